// Multicomponent form of the colour step: K <= 4 species on a rigid BCC
// lattice, one variance constraint per solute species.  Device structures
// shared by kernels_multi.cu and vcsgc_multi_capi.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "mlp.cuh"

namespace vcsgc {

constexpr int MK_MAX = 4;         // species
constexpr int MK_MAX_SH = 8;      // neighbour shells
constexpr int MK_MAX_OFF = 96;    // neighbour offsets (5 BCC shells: 58)
constexpr int MK_BLOCK = 128;
constexpr int MK_SCREEN_MAX_R = 1024;  // replicas of the screened form
constexpr uint32_t TAG_SPECIES = 6u;  // (step, domain rank): the proposed species

// Per-replica parameters: index alpha = 0..K-1, entry 0 (the solvent) zero.
struct MRepParams {
  double beta;
  double kappa_p[MK_MAX];
  double n0[MK_MAX];
  double dmu0[MK_MAX];  // phi_alpha + 2 kappa_p,alpha n0_alpha
  double phi[MK_MAX];
  uint2 key;
  // FP32 screen of the local decision (no re-embedding): beta, and
  // dF_ab + dmu0_b - dmu0_a rounded to float, [a K + b]
  float beta32;
  float c32[MK_MAX * MK_MAX];
  // the same with re-embedding: dmu0_b - dmu0_a rounded to float
  float cmu32[MK_MAX * MK_MAX];
};

struct MRepState {
  long long cnt[MK_MAX];
  long long step;
  long long fin_step;  // fused form: last step whose decision is folded in
  double energy;
  long long trials, local_acc, global_trials, global_acc, flips, near_ties, steps;
  double sum_c[MK_MAX], sum_c2[MK_MAX];
  long long s1_acc;  // delayed acceptance: trials that passed stage 1
};

// accumulator of one colour step (two per replica, by step parity)
struct MStepAcc {
  int dn[MK_MAX];
  int nacc;
  int ties;
  unsigned done;
  int accept;
  int s1;  // delayed acceptance: stage-1 passes
  double sum_de;
  // screened form: the species counts at the start of the step, written
  // with the zeroed sums by the commit of the step before (or the host), so
  // that every commit block can take the step's global decision
  long long cnt[MK_MAX];
};

struct MultiArgs {
  int R, K;
  int nx, ny, nz;
  long long N;
  // sublattice schedule: colour ((pz qy + py) qx + px) 2 + b
  int qx, qy, qz;
  int nxq, nyq, nzq;   // n / q per axis
  int n_colours;
  int D;               // trials per colour step (sites of one colour)
  // neighbour offsets in half-lattice units, sorted by shell
  int n_off, n_sh;
  int4 off[MK_MAX_OFF];  // (hx, hy, hz, shell)
  // shell tables: V[(s K + a) K + b] = phi_ab(r_s), Fd[s K + a] = f_a(r_s)
  const double* V;
  const double* Fd;
  int reembed;          // f_a(r_s) differs between species at some shell
  int bcc5;             // the offsets are the compile-time five-shell table
  const double* dF;     // [K][K] F_b(rho0) - F_a(rho0) (no re-embedding: rho uniform)
  // pair part in fixed point: Dq[((s K + a) K + b) K + beta] = round((phi_b,beta(r_s)
  // - phi_a,beta(r_s)) 2^qbits); sums of 58 such terms stay below 2^62
  const long long* Dq;
  int qbits;
  double qscale;        // 2^-qbits
  double inv_n;         // 1 / N (the per-step concentrations n / N)
  float rcp_nxq, rcp_nyq;  // 1 / nxq, 1 / nyq for the trial decode
  Spline embed[MK_MAX];
  uint8_t* types;       // [R][N]
  double* rho;          // [R][N]
  const MRepParams* rp;
  MRepState* rs;
  MStepAcc* acc;        // [R][3] (fused form: by step mod 3; else [R][2] by parity)
  int2* pend;           // [R][D] (site, new species) of the local accepts
  unsigned* err;
  // fused form (no re-embedding, five-shell table): one launch per colour
  // step.  A species byte carries the species in its low nibble and, while
  // a flip of the previous step awaits that step's global decision, the new
  // species + 1 in its high nibble.
  int fused;
  int* slot;            // [R][D] site of trial d's pending flip, or -1
  long long* nstart;    // [R][2][MK_MAX] counts at the start of a step, by parity
  const long long* base;  // step of launch j = 0
  // screened form (re-embedding, five-shell table): the local decision is
  // taken on an FP32 dE with a rigorous error bound, FP64 only where the
  // bound cannot decide.  The embedding cubics rounded to float
  // ([K][emb_n], one grid for all species), per site its density as a
  // float and the FP32 embedding value there, the largest error of one FP32
  // embedding evaluation (eV) and the argument range [emb_lo, emb_hi]
  // (the densities the lattice can reach) inside which that bound holds.
  int screen;
  const float4* emb32;
  int emb_n;
  float emb_ih;
  float emb_lo, emb_hi;
  float emb_err;
  // the table of species t holds F_t - F_t(rho_mid) (its coefficients'
  // rounding then scales with the offset values); emb_off[a K + b] =
  // F_b(rho_mid) - F_a(rho_mid) as a float, which an own-site change adds
  float emb_off[MK_MAX * MK_MAX];
  float qscale32;       // 2^-qbits as a float (exact)
  // (rho_i as float, the offset table's F32_{t_i} of that) per site,
  // [R][rf_n], laid out by
  // (basis, z, y, x mod qx, x div qx): the lanes of a warp, trials qx
  // cells apart along x, read neighbours at one offset from consecutive
  // entries.  rf_q = ceil(nx / qx); rf_n = 2 nz ny qx rf_q
  float2* rf;
  int rf_q;
  long long rf_n;
  int n_sm;             // multiprocessors of the device (commit grid)
  // delayed acceptance (K = 2, screened form): a trial first passes a
  // stage on the surrogate's prediction g of E(i = B) - E(i = A), then a
  // stage on the exact dE - s g.  The surrogate's descriptor comes from
  // nbc[R][rf_n] (laid out like rf): per site the B sites in each of its
  // five shells, 6 bits per shell (shell s at bit 6 s), kept up to date by
  // the commit while da is set.
  int da;
  MlpW mlp;
  uint32_t* nbc;
};

// site index of trial d of colour c (ascending site index within a colour)
__device__ __forceinline__ int multi_site(const MultiArgs& a, int c, int d) {
  const int b = c & 1;
  const int pc = c >> 1;
  const int px = pc % a.qx, py = (pc / a.qx) % a.qy, pz = pc / (a.qx * a.qy);
  const int kx = d % a.nxq, ky = (d / a.nxq) % a.nyq, kz = d / (a.nxq * a.nyq);
  const int cx = px + a.qx * kx, cy = py + a.qy * ky, cz = pz + a.qz * kz;
  return ((cz * a.ny + cy) * a.nx + cx) * 2 + b;
}

// lattice coordinates of site i: p = (2 cx + b, 2 cy + b, 2 cz + b)
__device__ __forceinline__ int3 multi_half(const MultiArgs& a, int i) {
  const int b = i & 1;
  const int cell = i >> 1;
  const int cx = cell % a.nx, cy = (cell / a.nx) % a.ny, cz = cell / (a.nx * a.ny);
  return make_int3(2 * cx + b, 2 * cy + b, 2 * cz + b);
}

// neighbour at half-lattice position p + h (periodic; |h| < 2 n per axis)
__device__ __forceinline__ int multi_nbr_at(const MultiArgs& a, int3 p, int4 h) {
  const int qx = p.x + h.x, qy = p.y + h.y, qz = p.z + h.z;
  const int bb = qx & 1;
  int X = (qx - bb) >> 1, Y = (qy - bb) >> 1, Z = (qz - bb) >> 1;
  X += X < 0 ? a.nx : (X >= a.nx ? -a.nx : 0);
  Y += Y < 0 ? a.ny : (Y >= a.ny ? -a.ny : 0);
  Z += Z < 0 ? a.nz : (Z >= a.nz ? -a.nz : 0);
  return ((Z * a.ny + Y) * a.nx + X) * 2 + bb;
}

// neighbour at half-lattice position p + h as cell (X, Y, Z) and basis bb
__device__ __forceinline__ void multi_nbr_cell(const MultiArgs& a, int3 p, int4 h, int& X, int& Y, int& Z, int& bb) {
  const int qx = p.x + h.x, qy = p.y + h.y, qz = p.z + h.z;
  bb = qx & 1;
  X = (qx - bb) >> 1;
  Y = (qy - bb) >> 1;
  Z = (qz - bb) >> 1;
  X += X < 0 ? a.nx : (X >= a.nx ? -a.nx : 0);
  Y += Y < 0 ? a.ny : (Y >= a.ny ? -a.ny : 0);
  Z += Z < 0 ? a.nz : (Z >= a.nz ? -a.nz : 0);
}

// entry of cell (X, Y, Z), basis b in the screened form's per-site floats
__device__ __forceinline__ long long multi_rfi(const MultiArgs& a, int X, int Y, int Z, int b) {
  const int xq = X / a.qx;
  return ((long long)(b * a.nz + Z) * a.ny + Y) * ((long long)a.qx * a.rf_q) + (long long)(X - xq * a.qx) * a.rf_q +
         xq;
}

__device__ __forceinline__ int multi_nbr(const MultiArgs& a, int i, int4 h) {
  return multi_nbr_at(a, multi_half(a, i), h);
}

// The 58 neighbours of a BCC site out to the fifth shell (r_c between
// a sqrt(3) and a sqrt(19)/2), as half-lattice offsets h (all even or all
// odd), ordered by |h|^2 then (hx, hy, hz): shells |h|^2 = 3, 4, 8, 11, 12
// with 8, 6, 12, 24, 8 sites.  Packed (hx + 4) | (hy + 4) << 4 |
// (hz + 4) << 8 | shell << 12; a compile-time switch so that unrolled
// loops fold the offsets into constants.
constexpr int MK_BCC5_N = 58;
__host__ __device__ __forceinline__ constexpr int mk_bcc5_code(int k) {
  switch (k) {
    case 0: return 0x0333; case 1: return 0x0533; case 2: return 0x0353; case 3: return 0x0553;
    case 4: return 0x0335; case 5: return 0x0535; case 6: return 0x0355; case 7: return 0x0555;
    case 8: return 0x1442; case 9: return 0x1424; case 10: return 0x1244; case 11: return 0x1644;
    case 12: return 0x1464; case 13: return 0x1446; case 14: return 0x2422; case 15: return 0x2242;
    case 16: return 0x2642; case 17: return 0x2462; case 18: return 0x2224; case 19: return 0x2624;
    case 20: return 0x2264; case 21: return 0x2664; case 22: return 0x2426; case 23: return 0x2246;
    case 24: return 0x2646; case 25: return 0x2466; case 26: return 0x3331; case 27: return 0x3531;
    case 28: return 0x3351; case 29: return 0x3551; case 30: return 0x3313; case 31: return 0x3513;
    case 32: return 0x3133; case 33: return 0x3733; case 34: return 0x3153; case 35: return 0x3753;
    case 36: return 0x3373; case 37: return 0x3573; case 38: return 0x3315; case 39: return 0x3515;
    case 40: return 0x3135; case 41: return 0x3735; case 42: return 0x3155; case 43: return 0x3755;
    case 44: return 0x3375; case 45: return 0x3575; case 46: return 0x3337; case 47: return 0x3537;
    case 48: return 0x3357; case 49: return 0x3557; case 50: return 0x4222; case 51: return 0x4622;
    case 52: return 0x4262; case 53: return 0x4662; case 54: return 0x4226; case 55: return 0x4626;
    case 56: return 0x4266; case 57: return 0x4666;
    default: return 0;
  }
}

void launch_multi_shell_tables(const Spline* pair, const Spline* dens, int K, const double* r_s, int n_sh,
                               double* V, double* Fd, unsigned* err, cudaStream_t st);
// dF[a K + b] = F_b(rho_0) - F_a(rho_0) at the uniform density rho_0 of site 0
void launch_multi_df(const MultiArgs& a, double* dF, cudaStream_t st);
void launch_multi_fixed(const double* V, int n_sh, int K, int qbits, long long* Dq, cudaStream_t st);
void launch_multi_rho(const MultiArgs& a, int r0, int nrep, cudaStream_t st);
// per-site energies summed into block partials part[r][blocks]
int multi_energy_blocks(long long N);
void launch_multi_energy(const MultiArgs& a, int r0, int nrep, double* part, cudaStream_t st);
void launch_multi_delta_e(const MultiArgs& a, int r, const long long* sites, const uint8_t* to, int n,
                          double* out, cudaStream_t st);
// delayed acceptance (K = 2, five-shell table): the per-site shell counts of
// every replica from its species; descriptors and exact targets of every
// site (rows r N + i) from those counts
void launch_multi_nbc(const MultiArgs& a, cudaStream_t st);
void launch_multi_features(const MultiArgs& a, float* X, float* Y, cudaStream_t st);
// one colour step (propose and commit); after_step: the previous launch on
// the stream is this context's commit (the screened form then overlaps).
// The screened form takes step *base + j (launch_multi_advance moves the
// base after a run of steps); the others keep the step in each replica's state.
void launch_multi_step(const MultiArgs& a, int j, cudaStream_t st, bool after_step);
// fused form: step base + j (propose = false: only the commit and the
// bookkeeping of the previous step), and base += n
void launch_multi_fused(const MultiArgs& a, int j, bool propose, cudaStream_t st);
void launch_multi_advance(long long* base, int n, cudaStream_t st);

}  // namespace vcsgc
