// kernels.h -- launchers of the device kernels (host-callable, internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "mlp.cuh"

namespace vcsgc {

constexpr int MC_BLOCK = 128;

// ---- tables (kernels_nbr.cu)
// Cubic coefficients of one table from knot values y[0..n) and optional knot
// derivatives m (nullptr: central differences); out has n-1 intervals.
void launch_spline_coeffs(const double* y, const double* m, int n, double h, Cubic* out,
                          cudaStream_t st);
// derivative quadratics (c1, 2 c2, 3 c3) / h of n_int cubic intervals
void launch_spline_derivs(const Cubic* c, int n_int, double h, Cubic* out, cudaStream_t st);
// coefficients rounded to float (mixed form)
void launch_to_cubic32(const Cubic* c, int n_int, Cubic32* out, cudaStream_t st);
// Per-shell pair and density differences of the rigid lattice:
// tab[0] = C_A, tab[1+s] = G_A[s], tab[1+S+s] = f_B(r_s) - f_A(r_s), tab[1+2S+s] = r_s,
// with r_s = (a/2) sqrt(h2[s]) and z[s] neighbours in shell s.
void launch_shell_tables(Tables tab, const int* h2, const int* z, int S, double a, double* out,
                         unsigned* err, cudaStream_t st, const Tables32* tab32 = nullptr);

// shell multiplicities passed by value
struct LatZ {
  int z[8];
};
// Energy table of the rigid lattice with uniform rho0 (kernels_nbr.cu):
// phi_AA, phi_AB, phi_BB at each shell radius, F_A(rho0), F_B(rho0), z_s
// (3 S + 2 + S doubles)
void launch_lattice_energy_table(Tables tab, const Tables32* tab32, const double* shell_tab, int S, LatZ z,
                                 const double* rho, double* etab, unsigned* err, cudaStream_t st);

// ---- neighbour lists (kernels_nbr.cu)
// Rigid BCC: row i lists the sites at the K half-lattice offsets hoff (x,y,z).
void launch_lattice_neighbours(int nx, int ny, int nz, const int3* hoff, int K, int* nbr, int* cnt,
                               cudaStream_t st);
// Explicit positions: cell binning (side >= rl, >= 3 cells per axis) and a
// full neighbour list within rl; rows longer than K set ERRF_OVERFLOW.
struct CellList {
  int nc[3];
  float* x32;      // [N] float copies of the positions (list criterion only)
  float* y32;
  float* z32;
  int* cell_of;    // [N]
  int* cell_count; // [ncell]
  int* cell_start; // [ncell + 1]
  int* cell_cursor;// [ncell]
  int* sorted;     // [N]
};
// Distance margin of the list's FP32 criterion: rows hold every pair within
// rl and may hold pairs up to rl + cell_list_margin(box).
inline double cell_list_margin(const double box[3]) {
  const double L = box[0] > box[1] ? (box[0] > box[2] ? box[0] : box[2]) : (box[1] > box[2] ? box[1] : box[2]);
  return 0.01 + 1e-6 * L;
}
void launch_cell_neighbours(long long N, const double* x, const double* y, const double* z,
                            const double box[3], double rl, CellList cl, int K, int* nbr, int* cnt,
                            unsigned* err, cudaStream_t st);
// SPATIAL colour schedule on the device: dom_start[ndom + 1] and
// dom_sites[N] (atoms by domain, ascending within one) from the positions;
// dom_of_block[nb0 nb1 nb2] gives each box's domain rank; dom_of[N],
// count[ndom] and cursor[ndom] are scratch
void launch_spatial_schedule(long long N, const double* x, const double* y, const double* z, const double box[3],
                             const int nb[3], const int* dom_of_block, int ndom, int* dom_of, int* count,
                             int* cursor, int* dom_start, int* dom_sites, cudaStream_t st);
// half list: the entries j > i of each full row (same stride K)
void launch_half_list(long long N, int K, const int* nbr, const int* cnt, int* nbr_h, int* cnt_h,
                      cudaStream_t st);

// ---- density, energy (kernels_nbr.cu)
// rho_i of replica r (shared array when !per_rep) and, if dF != nullptr,
// dF_i = F_B(rho_i) - F_A(rho_i).
void launch_rho(const McArgs& a, bool shell, int r, cudaStream_t st);
// screened re-embedding: per-site (float rho, F32 embedding) of replica r
void launch_fill_rf(const McArgs& a, int r, cudaStream_t st);
// Block partial sums of the energy of replica r into part[0..nblocks).
int energy_blocks(long long N);
void launch_energy(const McArgs& a, bool shell, int r, double* part, cudaStream_t st);

// ---- fused colour step of the rigid lattice (kernels_lattice.cu)
constexpr int LAT_BLOCK = 128;
constexpr int LAT_MAX_SH = 8;     // shells
constexpr int LAT_MAX_ROWS = 32;  // neighbour rows per basis
constexpr int LAT_HALO = 4;       // halo bits at each end of a row (>= hmax)

struct LatRow {
  int dy, dz;                   // row offset (cells) from the site's row
  uint32_t mask[LAT_MAX_SH];    // window bits of each shell
};

// per-replica constants of the FP32 screen of the local test
struct LatRep {
  float cpd32;   // C + dmu0 (eV)
  float beta32;  // 1/(kB T)
  float dx;      // absolute bound on |X32 - X| from the rounding of the inputs and sums
  float bk32;    // beta kappa_p (global stage)
  float n0_32;   // N c0
  float pad[3];
};

struct LatCtl {
  long long base_step;          // step of the next launch with j = 0
};

// colours and global uniforms of a chain's steps (entry j + 1: step
// base + j, j = -1 .. LAT_CTAB - 2), per replica
constexpr int LAT_CTAB = 65;

// geometry of one replica's rigid lattice in the bit-packed form
struct LatGeom {
  int nx, ny, nz, W;            // cells per axis, 64-bit words per row
  long long bits_off;           // first word of the replica's rows
  long long pend_off;           // first pending slot of the replica
  long long n_sites;
  int d;                        // domains per colour (SUBLATTICE)
  int dmax;                     // pending slots of the replica
  int nxq, nyq;                 // nx / qx, ny / qy
  float rcp_nx, rcp_ny, rcp_nxq, rcp_nyq;  // 1/d for fdiv
  long long site_off;           // first row of the replica in per-site outputs
};

struct LatArgs {
  int R;
  int block;                    // threads per block (64, 128 or 256)
  int prefetch;                 // load the trial's rows before the block barrier
  unsigned long long* bits;     // all replicas' rows (+1 pad word)
  const LatGeom* geom;          // [R]
  int hmax;                     // largest |half-lattice offset| along x
  int n_shells;                 // shells in use (<= LAT_MAX_SH)
  int n_rows[2];
  LatRow rows[2][LAT_MAX_ROWS];
  double C;                     // pair part of dE(A->B) with no B neighbour
  double G[LAT_MAX_SH];         // change per B neighbour in each shell
  float G32[LAT_MAX_SH];
  const double* dF;             // [N] F_B(rho_i) - F_A(rho_i) (single lattice)
  const float* dF32;            // [N] the same in FP32
  int df_uniform;               // every site has dF_i = dF0 (perfect lattice)
  double dF0;
  const LatRep* lrep;           // [R]
  // schedule
  int sublattice, qx, qy, qz;
  float rcp_qx, rcp_qy;
  int n_colours;
  const int* col_start;
  const int* dom_start;
  const int* dom_sites;
  PickTab pick;                 // site weights of overlapping domains (n = 0: uniform)
  int dmax;                     // largest pending-slot count of a replica
  const int2* blk;              // [n_blk] (replica, first trial) of each block of `block` threads
  int n_blk;
  // replicas
  const RepParams* rp;
  RepState* rs;
  StepAcc* acc;                 // [R][3]
  long long* n_start;           // [R][2]
  int* pend;                    // all replicas' pending slots
  LatCtl* ctl;
  int* ctab;                    // [R][LAT_CTAB]
  unsigned long long* ugtab;    // [R][LAT_CTAB] top 53 bits of the global uniform
  unsigned* err;
  // delayed acceptance (needs the 5-shell BCC neighbourhood): stage 1 tests
  // the surrogate's prediction, stage 2 the exact dE
  int da;
  MlpW mlp;
  int bcc5;                     // rows and masks equal the compile-time 5-shell BCC table
  int unpack4;                  // every replica's nx is even and its bytes 4-aligned: unpack 4 sites per thread
};

void launch_lattice_step(const LatArgs& a, int j, bool propose, cudaStream_t st);

// ---- cluster-resident form of the fused step (kernels_cluster.cu)
// Tiling of one replica's rows over the CTAs of its cluster: TY x TZ tiles
// (rank = tz TY + ty) of Ty rows by Tz planes (ny = TY Ty, nz = TZ Tz,
// Ty, Tz >= 2); lcap: accepted-trial list capacity per step (>= the trials
// of a CTA in a step).
struct ClTile {
  int TY, TZ, Ty, Tz, lcap;
};
constexpr int CL_TRIALS_PER_THREAD = 8;
// dynamic shared memory of a tile: rows with halo, one pad word (a trial's
// second window word may lie one past its row; its bits are never used),
// the uniforms of a step's trials, two accept lists
inline size_t cluster_smem_bytes(const ClTile& t, int W) {
  return sizeof(unsigned long long) * ((size_t)(t.Ty + 4) * (t.Tz + 4) * W + 1 + t.lcap) +
         sizeof(int) * 2 * (size_t)t.lcap;
}
// largest dynamic shared memory a tile may use
constexpr size_t CL_SMEM_MAX = 200 * 1024;
// n colour steps from step `base` of every replica (R clusters of `csize`
// CTAs of `block` threads, block 256 or 512); needs the five-shell table, the
// sublattice schedule, a uniform dF and no pending commit.  Returns the
// launch status.
cudaError_t launch_cluster_steps(const LatArgs& a, const ClTile* d_tiles, size_t smem, int csize, int block,
                                 long long base, int n, cudaStream_t st);
// clusters of csize CTAs with `smem` bytes each that can be resident at once
// (0: the shape cannot launch)
int cluster_capacity(int csize, int block, size_t smem);
// true when the rows and masks of a equal the compile-time five-shell table
bool lattice_rows_bcc5(const LatArgs& a);
// B count and energy of replicas r0 .. r0 + nrep - 1 from their packed
// species (perfect lattice, one density function; etab from
// launch_lattice_energy_table), written to their states (n, energy) and to
// n_start[2 r + parity]; part holds nrep * pstride * lattice_energy_width()
// doubles of scratch, pstride >= lattice_energy_blocks(max_words), max_words
// the largest replica's word count ny nz W
int lattice_energy_blocks(long long max_words);
int lattice_energy_width();
void launch_lattice_energy(const LatArgs& a, int r0, int nrep, long long max_words, const double* etab,
                           double* part, int pstride, int parity, cudaStream_t st);
// step base += n, then the colour table of the new base
void launch_lattice_advance(const LatArgs& a, int n, cudaStream_t st);
void launch_colour_table(const LatArgs& a, cudaStream_t st);
void launch_to_float(const double* in, float* out, long long n, cudaStream_t st);
// species bytes (tptr[r], a device array of R pointers) <-> bit rows of
// replicas r0 .. r0 + nrep - 1
void launch_lattice_pack(const LatArgs& a, uint8_t* const* tptr, int r0, int nrep, long long max_words,
                         cudaStream_t st);
// sets ERRF_SPECIES in *err when a byte of t[0..n) is neither 0 nor 1; the
// pack and lattice-energy kernels then write nothing
void launch_species_check(const uint8_t* t, long long n, unsigned* err, cudaStream_t st);
void launch_lattice_unpack(const LatArgs& a, uint8_t* const* tptr, int r0, int nrep, long long max_sites,
                           cudaStream_t st);
void launch_lattice_delta_e(const LatArgs& a, int r, const int* sites, int n, double* out, cudaStream_t st);
// Environment counts X[row][10] and exact targets Y[row] = E(i = B) - E(i = A)
// of every site of every replica (row = site_off + site); no pending flips.
void launch_lattice_features(const LatArgs& a, long long max_sites, float* X, float* Y, cudaStream_t st);

// ---- surrogate network (kernels_mlp.cu)
struct MlpBuf {
  uint2* w1f;   // [MLP_W1F]
  uint2* w2f;   // [MLP_W2F]
  uint2* w2tf;  // [MLP_W2F]
  float* vec;   // [MLP_VEC]
};
MlpW mlp_view(const MlpBuf& b);
void launch_mlp_pack(const float* p, const MlpBuf& b, cudaStream_t st);
void launch_mlp_forward(const MlpBuf& b, const float* X, long long n, float* out, cudaStream_t st);
// gradient of the mean squared error over a minibatch of B rows (sampled
// from the n rows by Philox(key, step = *ctr, row) when sample) added to grad;
// the batch loss is added to loss_hist[*ctr - *base] (loss_hist[0] when ctr
// is null)
void launch_mlp_backward(const MlpBuf& b, const float* X, const float* Y, long long n, long long B,
                         bool sample, uint2 key, const long long* ctr, const long long* base, float* grad,
                         double* loss_hist, cudaStream_t st);
// buffers of a surrogate object made by vcsgc_mlp_create (false if null)
bool mlp_object_buffers(void* mlp, MlpBuf* out);
cudaStream_t mlp_object_stream(void* mlp);
// one Adam step (learning rate lr decayed by a half cosine to lr / 100 over
// `total` steps counted from ctr[1]; no decay when total <= 1)
void launch_mlp_adam_pack(float* p, float* m, float* v, float* grad, float lr, long long total, long long* ctr,
                          const MlpBuf& b, cudaStream_t st);

// ---- colour step (kernels_mc.cu)
// phase 0: propose + commit; 1: propose only; 2: commit only
void launch_colour_step(const McArgs& a, bool shell, bool reembed, cudaStream_t st, int phase = 0);
void launch_delta_e_list(const McArgs& a, bool shell, bool reembed, int r, const int* sites, int n,
                         double* out, cudaStream_t st);

// ---- molecular dynamics (kernels_md.cu)
struct MdArgs {
  long long N;
  int K;
  const int* nbr;
  const int* nbr_cnt;
  const int* nbr_h;      // half list (j > i, stride K) of the FP64 form, or null
  const int* cnt_h;
  int same_dens;         // f_A = f_B: one density table value serves both ends
  const uint8_t* types;
  double *x, *y, *z, *vx, *vy, *vz, *fx, *fy, *fz;
  double* rho;
  double* dFp;   // F'(rho_i)
  float* dFp32;  // the same in FP32 (mixed form)
  double* dF;    // F_B(rho_i) - F_A(rho_i)
  double *x0, *y0, *z0;  // positions at the last neighbour build
  uint32_t *ux, *uy, *uz;  // fixed-point copies of x, y, z (mixed form; fix_diff)
  float ul[3];             // L 2^-32 per axis
  double box[3];
  double rc;
  double mass[2];
  double dt, c1, c2, kT;
  uint2 key;
  Tables tab;
  Tables32 tab32;
  int mixed;
  unsigned* err;
  unsigned long long* max_disp2_bits;  // max squared displacement (as bits)
  double* vir;   // accumulates the virial sum r_ij . F_ij (FP64 forms) when set
  double lam;    // box length over its length at the last neighbour build
};
// u = x / L 2^32 mod 2^32 per axis (fix_diff)
void launch_fix_positions(long long N, const double* x, const double* y, const double* z, const double box[3],
                          uint32_t* ux, uint32_t* uy, uint32_t* uz, cudaStream_t st);
// the mixed form refreshes the fixed-point positions first
void launch_md_rho(const MdArgs& m, cudaStream_t st);
void launch_md_force(const MdArgs& m, cudaStream_t st);
void launch_md_first_half(const MdArgs& m, long long md_step, cudaStream_t st);
void launch_md_second_half(const MdArgs& m, cudaStream_t st);
void launch_md_snapshot(const MdArgs& m, cudaStream_t st);
void launch_kinetic(const MdArgs& m, double* part, cudaStream_t st);
// Nose-Hoover / MTK sub-flows: v <- v s e1 + (F/m) he2; r <- r e1 + v e2dt
void launch_nh_kick(const MdArgs& m, double s, double e1, double he2, cudaStream_t st);
void launch_nh_drift(const MdArgs& m, double e1, double e2dt, cudaStream_t st);
// conjugate gradients: positions x0 + alpha d (SoA, 3N), dot-product block
// partials, max |a_i|^2 over atoms
void launch_cg_place(const MdArgs& m, const double* x0, const double* d, double alpha, cudaStream_t st);
int dot_blocks(long long n);
void launch_dot(const double* a, const double* b, long long n, double* part, cudaStream_t st);
void launch_max_norm2(const double* a, long long N, unsigned long long* out, cudaStream_t st);
// d <- g + beta d (n entries)
void launch_axpby(double* d, const double* g, double beta, long long n, cudaStream_t st);
int kinetic_blocks(long long N);

}  // namespace vcsgc
