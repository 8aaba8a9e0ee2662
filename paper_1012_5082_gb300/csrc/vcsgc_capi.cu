// vcsgc_capi.cu -- host side of the C ABI declared in include/vcsgc.h:
// argument checks, device allocation, table and schedule set-up, the
// graph-captured colour-step loop, the MD driver and the observables.
// Every numerical step of the method runs in the kernels of kernels_*.cu.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/vcsgc.h"
#include "common.cuh"
#include "kernels.h"
#include "multi_host.h"
#include "screen.h"
#include "trace.h"

using namespace vcsgc;

namespace {

std::string g_init_error;

struct Ctx {
  std::string err;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int device = 0;
  int kind = 0;
  int nx = 0, ny = 0, nz = 0;
  double a = 0;
  long long N = 0;
  double box[3] = {0, 0, 0};
  int R = 1;
  double rc = 0, skin = 0, rl = 0;
  bool shell = false, reembed = false;
  bool mixed = false;
  int sched_kind = 0;
  int sched[6] = {0, 0, 0, 0, 0, 0};
  long long steps_per_sweep = 1;
  // device memory
  std::vector<void*> allocs;
  uint8_t* types = nullptr;
  double* rho = nullptr;
  double* dF = nullptr;
  double* dFp = nullptr;
  float* dFp32 = nullptr;
  double *x = nullptr, *y = nullptr, *z = nullptr;
  double *vx = nullptr, *vy = nullptr, *vz = nullptr;
  double *fx = nullptr, *fy = nullptr, *fz = nullptr;
  double *x0 = nullptr, *y0 = nullptr, *z0 = nullptr;
  uint32_t *ux = nullptr, *uy = nullptr, *uz = nullptr;  // fixed-point positions (mixed, kind 1)
  unsigned long long* max_disp2 = nullptr;
  int* nbr = nullptr;
  int* nbr_cnt = nullptr;
  int K = 0;
  int* nbr_h = nullptr;            // half list of the FP64 MD form
  int* cnt_h = nullptr;
  int K_h = 0;                     // row stride nbr_h was allocated for
  Cubic* coef[7] = {};
  Cubic* dcoef[7] = {};
  double* shell_tab = nullptr;
  // screened re-embedding (rigid lattice): per-site floats, float cubics of
  // the embedding, the bound; the energy is recomputed when read
  bool screen = false;
  float2* rf = nullptr;
  float4* emb32 = nullptr;
  int emb_n = 0;
  float emb_ih = 0.f, emb_lo = 0.f, emb_hi = 0.f, emb_err = 0.f;
  bool energy_stale = false;
  int* col_start = nullptr;
  int* dom_start = nullptr;
  int* dom_sites = nullptr;
  long long dom_sites_cap = 0;     // entries dom_sites was allocated for
  PickTab pick{};                  // site weights of an OVERLAP schedule
  int n_colours = 0, dmax = 0;
  long long n_domains = 0;
  int sublattice_d = 0;            // domains per colour of a SUBLATTICE schedule
  RepParams* rp = nullptr;
  RepState* rs = nullptr;
  StepAcc* acc = nullptr;
  int* acc_list = nullptr;
  unsigned* derr = nullptr;
  double* part = nullptr;
  int part_n = 0;
  int* sites_buf = nullptr;
  double* de_buf = nullptr;
  int sites_cap = 0;
  CellList cl{};
  std::vector<RepParams> h_rp;
  // md
  bool have_v = false;
  long long md_step = 0;
  double mass[2] = {55.845, 63.546};
  double dt = 2.0, gamma = 0.01, T_md = 0.0;
  uint64_t md_seed = 0;
  bool forces_valid = false;
  // Nose-Hoover chains and the MTK barostat (kind 0: Langevin BAOAB)
  struct Nh {
    int kind = 0, chain = 3;
    double t_damp = 100.0, p_damp = 1000.0, p_ext = 0.0;  // fs, fs, eV/A^3
    double xi[4] = {}, eta[4] = {}, Q[4] = {}, xib[4] = {}, etab[4] = {}, Qb[4] = {};
    double veps = 0.0, W = 0.0;
    double vs = 1.0;  // velocity scale not yet applied on the device
  } nh;
  double* d_vir = nullptr;  // device accumulator of the virial
  double box_build[3] = {0, 0, 0};
  int ncell_cap = 0;
  // conjugate-gradient work vectors (SoA, 3N) and reduction partials
  double *cg_x0 = nullptr, *cg_d = nullptr, *cg_f = nullptr, *cg_g = nullptr, *cg_part = nullptr;
  // graph
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  McArgs mc{};
  MdArgs md{};
  // fused lattice form
  bool fast = false;
  bool no_fast = false;            // set-up only (sub-context of a batch)
  std::vector<LatGeom> h_geom;
  double df_absmax = 0.0, sum_absG = 0.0;
  // per-replica species arrays and sizes (single lattice: slices of types;
  // batch: the sub-contexts' arrays)
  std::vector<uint8_t*> rep_types;
  std::vector<long long> rep_n;
  std::vector<struct Ctx*> subs;   // batch of lattices of different sizes
  LatArgs lat{};
  long long h_base = 0;            // host mirror of lat.ctl->base_step
  bool pending = false;            // steps launched since the last flush
  void* h_pin = nullptr;           // pinned staging: RepState[R] then the error word
  size_t h_pin_bytes = 0;
  std::vector<int3> offsets;       // half-lattice neighbour offsets (kind 0)
  std::vector<int> offset_shell;
  // delayed acceptance: the context's copy of the surrogate's fragments
  MlpBuf sur{};
  // fused form, perfect lattice: energy table and partial sums of the
  // lattice energy kernel (species set from the host)
  double* etab = nullptr;
  double* epart = nullptr;
  int epstride = 0;                // lattice-energy partials per replica
  uint8_t** d_tptr = nullptr;      // device array of the replicas' species arrays
  long long max_words = 0, max_sites = 0;
  // fused form: block tables for blocks of 64, 128, 256 threads
  int2* blk_tab[3] = {nullptr, nullptr, nullptr};
  int n_blk_tab[3] = {0, 0, 0};
  // cluster-resident form (launch form 1): per cluster size 1, 2, 4, 8, 16
  // the replicas' tilings on the device (null: that size cannot serve every
  // replica) and the shared memory a CTA needs
  int form = 0;
  int cl_size = 0, cl_block = 512;
  ClTile* cl_tiles[5] = {};
  size_t cl_smem[5] = {};
  int cl_lcap[5] = {};             // most trials of one CTA in one step
  long long base_lag = 0;          // steps run in form 1 not yet added to lat.ctl->base_step
  // SPATIAL schedule rebuilt on the device between MD phases: box -> domain
  // rank, and scratch of the counting sort
  int* sp_dom_of_block = nullptr;
  int* sp_dom_of = nullptr;
  int* sp_count = nullptr;
  int* sp_cursor = nullptr;
  int sp_ndom = 0;
  // species-dependent densities on the period-q sublattice: the colour steps
  // run through a two-species multicomponent object (its FP32-screened
  // kernels with compile-time offsets); this context mirrors its species and
  // running state on reading
  void* multi = nullptr;
  bool multi_dirty = false;
};

// index of a cluster size in Ctx::cl_tiles (-1: not a supported size)
int cl_index(int csize) {
  switch (csize) {
    case 1: return 0;
    case 2: return 1;
    case 4: return 2;
    case 8: return 3;
    case 16: return 4;
    default: return -1;
  }
}

// point the fused step at the block table of its block size
void select_blk(Ctx* c) {
  const int q = c->lat.block == 64 ? 0 : (c->lat.block == 256 ? 2 : 1);
  c->lat.blk = c->blk_tab[q];
  c->lat.n_blk = c->n_blk_tab[q];
}

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      c->err = std::string(#call) + ": " + cudaGetErrorString(e_);                     \
      return VCSGC_ERR_CUDA;                                                           \
    }                                                                                  \
  } while (0)

int flush(Ctx* c);
int sync_bytes(Ctx* c, int r);
int sync_from_multi(Ctx* c);

int fail(Ctx* c, int code, const std::string& msg) {
  c->err = msg;
  return code;
}

template <typename T>
int dalloc(Ctx* c, T** p, size_t count) {
  void* q = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(&q, sizeof(T) * count);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, VCSGC_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  c->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return VCSGC_OK;
}

#define TRY(expr)             \
  do {                        \
    int rc_ = (expr);         \
    if (rc_ != VCSGC_OK) return rc_; \
  } while (0)

// the device error bits e (already copied to the host) as a status
int device_error_status(Ctx* c, unsigned e) {
  if (!e) return VCSGC_OK;
  CK(cudaMemsetAsync(c->derr, 0, sizeof(unsigned), c->st));
  CK(cudaStreamSynchronize(c->st));
  if (e & ERRF_SPECIES) return fail(c, VCSGC_ERR_INVALID_ARG, "species must be 0 or 1");
  if (e & ERRF_TIMEOUT) return fail(c, VCSGC_ERR_TIMEOUT, "a bounded device wait ran out");
  if (e & ERRF_OVERFLOW) return fail(c, VCSGC_ERR_OVERFLOW, "neighbour list capacity exceeded");
  if (e & ERRF_TABLE) return fail(c, VCSGC_ERR_TABLE_RANGE, "r or rho outside the EAM table grid");
  return fail(c, VCSGC_ERR_NONFINITE, "non-finite energy difference or force");
}

int check_device_error(Ctx* c) {
  unsigned e = 0;
  CK(cudaMemcpyAsync(&e, c->derr, sizeof(unsigned), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return device_error_status(c, e);
}

void fill_args(Ctx* c) {
  McArgs& a = c->mc;
  a.N = c->N;
  a.R = c->R;
  a.K = c->K;
  a.nbr = c->nbr;
  a.nbr_cnt = c->nbr_cnt;
  a.types = c->types;
  a.rho = c->rho;
  a.rho_per_rep = c->reembed ? 1 : 0;
  a.dF = c->dF;
  a.vel[0] = c->have_v ? c->vx : nullptr;
  a.vel[1] = c->have_v ? c->vy : nullptr;
  a.vel[2] = c->have_v ? c->vz : nullptr;
  a.mass[0] = c->mass[0];
  a.mass[1] = c->mass[1];
  a.shell_tab = c->shell_tab;
  a.x = c->x;
  a.y = c->y;
  a.z = c->z;
  a.ux = c->ux;
  a.uy = c->uy;
  a.uz = c->uz;
  for (int q = 0; q < 3; ++q) {
    a.box[q] = c->box[q];
    a.ul[q] = (float)(c->box[q] * 0x1p-32);
  }
  a.rc = c->rc;
  a.mixed = c->mixed ? 1 : 0;
  a.screen = c->screen ? 1 : 0;
  a.rf = c->rf;
  a.emb32 = c->emb32;
  a.emb_n = c->emb_n;
  a.emb_ih = c->emb_ih;
  a.emb_lo = c->emb_lo;
  a.emb_hi = c->emb_hi;
  a.emb_err = c->emb_err;
  a.n_colours = c->n_colours;
  a.col_start = c->col_start;
  a.dom_start = c->dom_start;
  a.dom_sites = c->dom_sites;
  a.pick = c->pick;
  a.dmax = c->dmax;
  a.rp = c->rp;
  a.rs = c->rs;
  a.acc = c->acc;
  a.acc_list = c->acc_list;
  a.err = c->derr;

  MdArgs& m = c->md;
  m.N = c->N;
  m.K = c->K;
  m.nbr = c->nbr;
  m.nbr_cnt = c->nbr_cnt;
  m.nbr_h = c->K_h == c->K ? c->nbr_h : nullptr;
  m.cnt_h = c->cnt_h;
  m.same_dens = c->reembed ? 0 : 1;
  m.types = c->types;
  m.x = c->x; m.y = c->y; m.z = c->z;
  m.vx = c->vx; m.vy = c->vy; m.vz = c->vz;
  m.fx = c->fx; m.fy = c->fy; m.fz = c->fz;
  m.rho = c->rho;
  m.dFp = c->dFp;
  m.dF = c->dF;
  m.x0 = c->x0; m.y0 = c->y0; m.z0 = c->z0;
  m.ux = c->ux; m.uy = c->uy; m.uz = c->uz;
  for (int q = 0; q < 3; ++q) {
    m.box[q] = c->box[q];
    m.ul[q] = (float)(c->box[q] * 0x1p-32);
  }
  m.rc = c->rc;
  m.mass[0] = c->mass[0];
  m.mass[1] = c->mass[1];
  m.dt = c->dt;
  m.c1 = std::exp(-c->gamma * c->dt);
  m.c2 = std::sqrt(std::max(0.0, 1.0 - m.c1 * m.c1));
  m.kT = KB_EV * c->T_md;
  m.key = make_uint2((uint32_t)c->md_seed, (uint32_t)(c->md_seed >> 32));
  m.tab = c->mc.tab;
  m.tab32 = c->mc.tab32;
  m.mixed = c->mixed ? 1 : 0;
  m.dFp32 = c->dFp32;
  m.err = c->derr;
  m.max_disp2_bits = c->max_disp2;
  m.vir = c->d_vir;
  m.lam = c->box_build[0] > 0.0 ? c->box[0] / c->box_build[0] : 1.0;

  LatArgs& l = c->lat;
  l.R = c->R;
  l.sublattice = c->sched_kind == VCSGC_SCHED_SUBLATTICE ? 1 : 0;
  l.qx = c->sched[0];
  l.qy = c->sched[1];
  l.qz = c->sched[2];
  l.n_colours = c->n_colours;
  l.col_start = c->col_start;
  l.dom_start = c->dom_start;
  l.dom_sites = c->dom_sites;
  l.pick = c->pick;
  l.rp = c->rp;
  l.rs = c->rs;
  l.err = c->derr;
}

void drop_graph(Ctx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
  c->graph_steps = 0;
}

// ----------------------------------------------------------- neighbours
int build_cell_list(Ctx* c) {
  for (int q = 0; q < 3; ++q) {
    c->cl.nc[q] = (int)std::floor(c->box[q] / c->rl);
    if (c->cl.nc[q] < 3 || c->box[q] <= 2.0 * c->rl)
      return fail(c, VCSGC_ERR_STATE, "box no longer exceeds 2 (r_c + skin) with 3 cells");
    c->box_build[q] = c->box[q];
  }
  const int ncell = c->cl.nc[0] * c->cl.nc[1] * c->cl.nc[2];
  if (!c->cl.cell_of) {
    TRY(dalloc(c, &c->cl.x32, c->N));
    TRY(dalloc(c, &c->cl.y32, c->N));
    TRY(dalloc(c, &c->cl.z32, c->N));
    TRY(dalloc(c, &c->cl.cell_of, c->N));
    TRY(dalloc(c, &c->cl.sorted, c->N));
  }
  if (ncell > c->ncell_cap) {
    // the box can grow under a barostat
    TRY(dalloc(c, &c->cl.cell_count, ncell));
    TRY(dalloc(c, &c->cl.cell_start, ncell + 1));
    TRY(dalloc(c, &c->cl.cell_cursor, ncell));
    c->ncell_cap = ncell;
  }
  for (int attempt = 0; attempt < 6; ++attempt) {
    CK(cudaMemsetAsync(c->derr, 0, sizeof(unsigned), c->st));
    launch_cell_neighbours(c->N, c->x, c->y, c->z, c->box, c->rl, c->cl, c->K, c->nbr, c->nbr_cnt,
                           c->derr, c->st);
    CK(cudaGetLastError());
    unsigned e = 0;
    CK(cudaMemcpyAsync(&e, c->derr, sizeof(unsigned), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (!(e & ERRF_OVERFLOW)) {
      if (c->R == 1) {
        // half list for the MD passes (each pair once)
        if (c->K_h != c->K) {
          TRY(dalloc(c, &c->nbr_h, (size_t)c->N * c->K));
          if (!c->cnt_h) TRY(dalloc(c, &c->cnt_h, c->N));
          c->K_h = c->K;
          fill_args(c);
        }
        launch_half_list(c->N, c->K, c->nbr, c->nbr_cnt, c->nbr_h, c->cnt_h, c->st);
        CK(cudaGetLastError());
      }
      return VCSGC_OK;
    }
    // grow the rows and rebuild
    const int K2 = ((c->K * 3 / 2) + 7) / 8 * 8;
    int* nb = nullptr;
    TRY(dalloc(c, &nb, (size_t)c->N * K2));
    c->nbr = nb;
    c->K = K2;
    fill_args(c);
    drop_graph(c);
  }
  return fail(c, VCSGC_ERR_OVERFLOW, "neighbour rows kept overflowing");
}

// ------------------------------------------------------------- schedule
// Host tables of the colour schedule: col_start[n_colours+1] indexes
// domains, dom_start[n_domains+1] indexes dom_sites; wt (OVERLAP only) holds
// each entry's pick weight.
struct Sched {
  std::vector<int> col, dom, sites, wt;
};

double cell_gap_distance(double a, int gap_cells) {
  // closest BCC pair across gap_cells empty cells: a corner site and a
  // body-centre site, a*sqrt((gap + 1/2)^2 + 1/2)
  const double g = gap_cells + 0.5;
  return a * std::sqrt(g * g + 0.5);
}

int build_schedule(Ctx* c, const std::vector<double>& hx, const std::vector<double>& hy,
                   const std::vector<double>& hz, Sched& S) {
  const double two_rc = 2.0 * c->rc;
  const int* p = c->sched;
  if (c->sched_kind == VCSGC_SCHED_BLOCKS || c->sched_kind == VCSGC_SCHED_SUBLATTICE ||
      c->sched_kind == VCSGC_SCHED_OVERLAP) {
    if (c->kind != 0) return fail(c, VCSGC_ERR_INVALID_ARG, "lattice schedules need a rigid lattice");
  }
  if (c->sched_kind == VCSGC_SCHED_BLOCKS) {
    const int bx = p[0], by = p[1], bz = p[2], px = p[3], py = p[4], pz = p[5];
    if (bx < 1 || by < 1 || bz < 1 || px < 1 || py < 1 || pz < 1 || c->nx % bx || c->ny % by || c->nz % bz)
      return fail(c, VCSGC_ERR_SCHEDULE, "block size does not divide the lattice");
    const int nbx = c->nx / bx, nby = c->ny / by, nbz = c->nz / bz;
    if (nbx % px || nby % py || nbz % pz) return fail(c, VCSGC_ERR_SCHEDULE, "colour period does not divide the blocks");
    const int nb[3] = {nbx, nby, nbz}, pp[3] = {px, py, pz}, bb[3] = {bx, by, bz};
    for (int q = 0; q < 3; ++q)
      if (nb[q] > pp[q] && cell_gap_distance(c->a, (pp[q] - 1) * bb[q]) <= two_rc)
        return fail(c, VCSGC_ERR_SCHEDULE, "same-colour blocks closer than 2 r_c");
    const int ncol = px * py * pz;
    S.col.assign(ncol + 1, 0);
    for (int col = 0; col < ncol; ++col) {
      S.col[col] = (int)S.dom.size();
      for (int ibz = 0; ibz < nbz; ++ibz)
        for (int iby = 0; iby < nby; ++iby)
          for (int ibx = 0; ibx < nbx; ++ibx) {
            if (((ibz % pz) * py + (iby % py)) * px + (ibx % px) != col) continue;
            S.dom.push_back((int)S.sites.size());
            for (int lz = 0; lz < bz; ++lz)
              for (int ly = 0; ly < by; ++ly)
                for (int lx = 0; lx < bx; ++lx)
                  for (int b = 0; b < 2; ++b) {
                    const long long cx = ibx * bx + lx, cy = iby * by + ly, cz = ibz * bz + lz;
                    S.sites.push_back((int)(((cz * c->ny + cy) * c->nx + cx) * 2 + b));
                  }
          }
    }
    S.col[ncol] = (int)S.dom.size();
    S.dom.push_back((int)S.sites.size());
  } else if (c->sched_kind == VCSGC_SCHED_SUBLATTICE) {
    const int qx = p[0], qy = p[1], qz = p[2];
    if (qx < 1 || qy < 1 || qz < 1 || c->nx % qx || c->ny % qy || c->nz % qz)
      return fail(c, VCSGC_ERR_SCHEDULE, "sublattice period does not divide the lattice");
    const int n3[3] = {c->nx, c->ny, c->nz}, q3[3] = {qx, qy, qz};
    for (int q = 0; q < 3; ++q)
      if (n3[q] > q3[q] && q3[q] * c->a <= two_rc)
        return fail(c, VCSGC_ERR_SCHEDULE, "same-colour sublattice sites closer than 2 r_c");
    const int ncol = qx * qy * qz * 2;
    // bucket the sites by colour, ascending site index within a colour
    std::vector<int> count(ncol + 1, 0);
    auto colour_of = [&](long long i) {
      const long long b = i & 1, cell = i >> 1;
      const long long cx = cell % c->nx, cy = (cell / c->nx) % c->ny, cz = cell / ((long long)c->nx * c->ny);
      return (int)((((cz % qz) * qy + (cy % qy)) * qx + (cx % qx)) * 2 + b);
    };
    for (long long i = 0; i < c->N; ++i) count[colour_of(i) + 1]++;
    for (int q = 0; q < ncol; ++q) count[q + 1] += count[q];
    S.col = count;
    S.sites.assign(c->N, 0);
    std::vector<int> cur(count.begin(), count.end() - 1);
    for (long long i = 0; i < c->N; ++i) S.sites[cur[colour_of(i)]++] = (int)i;
    S.dom.resize(c->N + 1);
    for (long long i = 0; i <= c->N; ++i) S.dom[i] = (int)i;
  } else if (c->sched_kind == VCSGC_SCHED_OVERLAP) {
    // cells of l lattice cells per axis; the domain of colour bit b covers
    // cell-local coordinates [b g, b g + l - g); weight 8 / coverage
    const int n3[3] = {c->nx, c->ny, c->nz};
    int l3[3], g3[3], nc[3], ld[3];
    for (int q = 0; q < 3; ++q) {
      l3[q] = p[q];
      g3[q] = p[3 + q];
      if (l3[q] < 1 || g3[q] < 0 || 2 * g3[q] > l3[q] || n3[q] % l3[q])
        return fail(c, VCSGC_ERR_SCHEDULE, "overlap cells do not divide the lattice, or 2 g > l");
      nc[q] = n3[q] / l3[q];
      ld[q] = l3[q] - g3[q];
      if (nc[q] > 1 && cell_gap_distance(c->a, g3[q]) <= two_rc)
        return fail(c, VCSGC_ERR_SCHEDULE, "same-colour overlapping domains closer than 2 r_c");
    }
    // coverage of a cell-local coordinate along one axis: 1 or 2
    auto cover = [&](int q, int x) { return (x < ld[q] ? 1 : 0) + (x >= g3[q] ? 1 : 0); };
    const long long per_dom = 2LL * ld[0] * ld[1] * ld[2];
    const long long ncell = (long long)nc[0] * nc[1] * nc[2];
    if (8 * ncell * per_dom >= (1LL << 31)) return fail(c, VCSGC_ERR_SCHEDULE, "overlap tables too large");
    S.col.assign(9, 0);
    std::vector<int> tmp, tw;
    for (int col = 0; col < 8; ++col) {
      const int o[3] = {(col & 1) * g3[0], ((col >> 1) & 1) * g3[1], ((col >> 2) & 1) * g3[2]};
      S.col[col] = (int)S.dom.size();
      for (int icz = 0; icz < nc[2]; ++icz)
        for (int icy = 0; icy < nc[1]; ++icy)
          for (int icx = 0; icx < nc[0]; ++icx) {
            tmp.clear();
            tw.clear();
            for (int tz = o[2]; tz < o[2] + ld[2]; ++tz)
              for (int ty = o[1]; ty < o[1] + ld[1]; ++ty)
                for (int tx = o[0]; tx < o[0] + ld[0]; ++tx) {
                  const long long cx = (long long)icx * l3[0] + tx, cy = (long long)icy * l3[1] + ty,
                                  cz = (long long)icz * l3[2] + tz;
                  const int w = 8 / (cover(0, tx) * cover(1, ty) * cover(2, tz));
                  for (int b = 0; b < 2; ++b) {
                    tmp.push_back((int)(((cz * c->ny + cy) * c->nx + cx) * 2 + b));
                    tw.push_back(w);
                  }
                }
            S.dom.push_back((int)S.sites.size());
            for (int w = 8; w >= 1; w >>= 1)
              for (size_t q = 0; q < tmp.size(); ++q)
                if (tw[q] == w) {
                  S.sites.push_back(tmp[q]);
                  S.wt.push_back(w);
                }
          }
    }
    S.col[8] = (int)S.dom.size();
    S.dom.push_back((int)S.sites.size());
  } else if (c->sched_kind == VCSGC_SCHED_SPATIAL) {
    const int nb[3] = {p[0], p[1], p[2]}, pp[3] = {p[3], p[4], p[5]};
    for (int q = 0; q < 3; ++q) {
      if (nb[q] < 1 || pp[q] < 1 || nb[q] % pp[q]) return fail(c, VCSGC_ERR_SCHEDULE, "spatial blocks do not divide");
      if (nb[q] > pp[q] && (pp[q] - 1) * c->box[q] / nb[q] <= two_rc)
        return fail(c, VCSGC_ERR_SCHEDULE, "same-colour spatial blocks closer than 2 r_c");
    }
    const int nblk = nb[0] * nb[1] * nb[2];
    const int ncol = pp[0] * pp[1] * pp[2];
    auto cidx = [](double v, double L, int n) {
      int q = (int)std::floor(v / L * n);
      return q < 0 ? 0 : (q >= n ? n - 1 : q);
    };
    std::vector<int> blk(c->N);
    std::vector<int> bcount(nblk + 1, 0);
    for (long long i = 0; i < c->N; ++i) {
      blk[i] = (cidx(hz[i], c->box[2], nb[2]) * nb[1] + cidx(hy[i], c->box[1], nb[1])) * nb[0] +
               cidx(hx[i], c->box[0], nb[0]);
      bcount[blk[i] + 1]++;
    }
    // domains ordered by colour, then block index; sites ascending
    std::vector<int> order;
    S.col.assign(ncol + 1, 0);
    for (int col = 0; col < ncol; ++col) {
      S.col[col] = (int)order.size();
      for (int b = 0; b < nblk; ++b) {
        const int ibx = b % nb[0], iby = (b / nb[0]) % nb[1], ibz = b / (nb[0] * nb[1]);
        if (((ibz % pp[2]) * pp[1] + (iby % pp[1])) * pp[0] + (ibx % pp[0]) == col) order.push_back(b);
      }
    }
    S.col[ncol] = (int)order.size();
    for (int b = 0; b < nblk; ++b) bcount[b + 1] += bcount[b];
    std::vector<int> by_blk(c->N);
    std::vector<int> cur(bcount.begin(), bcount.end() - 1);
    for (long long i = 0; i < c->N; ++i) by_blk[cur[blk[i]]++] = (int)i;
    S.dom.clear();
    S.sites.clear();
    S.sites.reserve(c->N);
    for (int b : order) {
      S.dom.push_back((int)S.sites.size());
      for (int q = bcount[b]; q < bcount[b + 1]; ++q) S.sites.push_back(by_blk[q]);
    }
    S.dom.push_back((int)S.sites.size());
  } else {
    return fail(c, VCSGC_ERR_INVALID_ARG, "unknown schedule");
  }
  return VCSGC_OK;
}

// Class table of the weighted pick: every domain must list the same
// sequence of weights (true of the OVERLAP geometry), each a power of two.
static int pick_table(Ctx* c, const Sched& S, PickTab& t) {
  t = PickTab{};
  if (S.wt.empty()) return VCSGC_OK;
  const int n0 = S.dom[1] - S.dom[0];
  for (int k = 0; k < n0;) {
    const int w = S.wt[k];
    int e = k;
    while (e < n0 && S.wt[e] == w) ++e;
    if (t.n == 4 || w < 1 || (w & (w - 1))) return fail(c, VCSGC_ERR_SCHEDULE, "pick weights not in four power-of-two classes");
    t.beg[t.n] = k;
    t.sh[t.n] = __builtin_ctz((unsigned)w);
    t.cum[t.n] = (t.n ? t.cum[t.n - 1] : 0) + (e - k) * w;
    ++t.n;
    k = e;
  }
  for (size_t d = 0; d + 1 < S.dom.size(); ++d) {
    if (S.dom[d + 1] - S.dom[d] != n0) return fail(c, VCSGC_ERR_SCHEDULE, "weighted domains differ in size");
    for (int k = 0; k < n0; ++k)
      if (S.wt[S.dom[d] + k] != S.wt[k]) return fail(c, VCSGC_ERR_SCHEDULE, "weighted domains differ in weights");
  }
  return VCSGC_OK;
}

int upload_schedule(Ctx* c, const Sched& S) {
  const int ncol = (int)S.col.size() - 1;
  int dmax = 0;
  for (int q = 0; q < ncol; ++q) dmax = std::max(dmax, S.col[q + 1] - S.col[q]);
  TRY(pick_table(c, S, c->pick));
  const bool realloc_needed = !c->col_start || ncol != c->n_colours ||
                              (long long)S.dom.size() - 1 != c->n_domains || dmax > c->dmax;
  if (realloc_needed) {
    TRY(dalloc(c, &c->col_start, S.col.size()));
    TRY(dalloc(c, &c->dom_start, S.dom.size()));
    if (dmax > c->dmax) TRY(dalloc(c, &c->acc_list, (size_t)c->R * dmax));
    drop_graph(c);
  }
  if ((long long)S.sites.size() > c->dom_sites_cap) {
    TRY(dalloc(c, &c->dom_sites, S.sites.size()));
    c->dom_sites_cap = (long long)S.sites.size();
    drop_graph(c);
  }
  CK(cudaMemcpyAsync(c->col_start, S.col.data(), sizeof(int) * S.col.size(), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->dom_start, S.dom.data(), sizeof(int) * S.dom.size(), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->dom_sites, S.sites.data(), sizeof(int) * S.sites.size(), cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  c->n_colours = ncol;
  c->n_domains = (long long)S.dom.size() - 1;
  c->dmax = std::max(c->dmax, dmax);
  const int dpc = S.col[1] - S.col[0];
  c->steps_per_sweep = dpc > 0 ? std::max(1LL, (c->N + dpc / 2) / dpc) : 1;
  c->sublattice_d = c->sched_kind == VCSGC_SCHED_SUBLATTICE ? dpc : 0;
  fill_args(c);
  return VCSGC_OK;
}

int positions_host(Ctx* c, std::vector<double>& hx, std::vector<double>& hy, std::vector<double>& hz) {
  hx.resize(c->N);
  hy.resize(c->N);
  hz.resize(c->N);
  CK(cudaMemcpyAsync(hx.data(), c->x, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(hy.data(), c->y, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(hz.data(), c->z, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return VCSGC_OK;
}

// --------------------------------------------------------------- energy
int energy_of(Ctx* c, int r, double* out) {
  TRY(sync_bytes(c, r));
  if (!c->subs.empty()) {
    CK(cudaStreamSynchronize(c->st));
    const int rc = energy_of(c->subs[r], 0, out);
    if (rc != VCSGC_OK) c->err = c->subs[r]->err;
    return rc;
  }
  launch_energy(c->mc, c->shell, r, c->part, c->st);
  CK(cudaGetLastError());
  std::vector<double> h(c->part_n);
  CK(cudaMemcpyAsync(h.data(), c->part, sizeof(double) * c->part_n, cudaMemcpyDeviceToHost, c->st));
  TRY(check_device_error(c));
  // compensated sum of the block partials
  double s = 0.0, comp = 0.0;
  for (double v : h) {
    const double t = s + v;
    comp += std::fabs(s) >= std::fabs(v) ? (s - t) + v : (v - t) + s;
    s = t;
  }
  *out = s + comp;
  return VCSGC_OK;
}

// recompute rho (and dF) of replica r, or of the shared array
int refresh_rho(Ctx* c, int r) {
  launch_rho(c->mc, c->shell, r, c->st);
  if (c->screen) launch_fill_rf(c->mc, r, c->st);
  CK(cudaGetLastError());
  return VCSGC_OK;
}

// screened form: the tracked energies are not kept up to date by the sweep;
// recompute them before anything reads the replica states
int refresh_energies(Ctx* c) {
  if (!c->screen || !c->energy_stale) return VCSGC_OK;
  for (int r = 0; r < c->R; ++r) {
    double e;
    TRY(energy_of(c, r, &e));
    CK(cudaMemcpyAsync(&c->rs[r].energy, &e, sizeof(double), cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
  }
  c->energy_stale = false;
  return VCSGC_OK;
}

// Tables and bound of the screened re-embedding form (rigid lattice, shell
// form; the bound: screen.h)
int screen_setup(Ctx* c) {
  const int n = c->mc.tab.sp[5].n_int;
  const double h = 1.0 / c->mc.tab.sp[5].inv_h;
  if (c->mc.tab.sp[6].n_int != n || c->mc.tab.sp[6].inv_h != c->mc.tab.sp[5].inv_h) return VCSGC_OK;
  TRY(dalloc(c, &c->emb32, (size_t)2 * n));
  std::vector<std::vector<Cubic>> hc(2, std::vector<Cubic>((size_t)n));
  for (int t = 0; t < 2; ++t) {
    launch_to_cubic32(c->coef[5 + t], n, reinterpret_cast<Cubic32*>(c->emb32 + (size_t)t * n), c->st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(hc[t].data(), c->coef[5 + t], sizeof(Cubic) * n, cudaMemcpyDeviceToHost, c->st));
  }
  const int S = c->mc.n_shells;
  std::vector<double> dfs((size_t)S);
  CK(cudaMemcpyAsync(dfs.data(), c->shell_tab + 1 + S, sizeof(double) * S, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  double dmax = 0.0;
  for (double v : dfs) dmax = std::max(dmax, std::fabs(v));
  const ScreenBound sb = screen_bound(hc, h, dmax);
  if (!std::isfinite(sb.err)) return fail(c, VCSGC_ERR_NONFINITE, "non-finite embedding table");
  TRY(dalloc(c, &c->rf, (size_t)c->R * c->N));
  c->emb_n = n;
  c->emb_ih = (float)c->mc.tab.sp[5].inv_h;
  c->emb_lo = (float)sb.lo;
  c->emb_hi = (float)sb.hi;
  c->emb_err = (float)sb.err;
  c->screen = true;
  fill_args(c);
  return VCSGC_OK;
}

int sync_state_from_types(Ctx* c, int r, const uint8_t* host_types) {
  long long nb = 0;
  for (long long i = 0; i < c->N; ++i) nb += host_types[i];
  if (c->reembed || r == 0) TRY(refresh_rho(c, r));
  double e = 0.0;
  TRY(energy_of(c, r, &e));
  RepState s;
  CK(cudaMemcpyAsync(&s, c->rs + r, sizeof(RepState), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  s.n = nb;
  s.energy = e;
  CK(cudaMemcpyAsync(c->rs + r, &s, sizeof(RepState), cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  return VCSGC_OK;
}

// bring the device step base (and the colour table of the per-step launch)
// up to the host's after steps run in the cluster-resident form
int sync_base(Ctx* c) {
  if (c->base_lag == 0) return VCSGC_OK;
  launch_lattice_advance(c->lat, (int)c->base_lag, c->st);
  CK(cudaGetLastError());
  c->base_lag = 0;
  return VCSGC_OK;
}

bool cluster_form_usable(const Ctx* c) {
  const int q = cl_index(c->cl_size);
  return c->form == 1 && q >= 0 && c->cl_tiles[q] && !c->lat.da;
}

// n colour steps in the cluster-resident form: any pending commit of the
// per-step form first, then one persistent launch per chunk of steps
int run_steps_cluster(Ctx* c, long long n) {
  TRY(flush(c));
  const int q = cl_index(c->cl_size);
  const long long chunk = 1LL << 20;
  while (n > 0) {
    const int m = (int)std::min(n, chunk);
    CK(launch_cluster_steps(c->lat, c->cl_tiles[q], c->cl_smem[q], c->cl_size, c->cl_block, c->h_base, m, c->st));
    c->h_base += m;
    c->base_lag += m;
    n -= m;
  }
  c->pending = false;
  return VCSGC_OK;
}

int run_steps_fast(Ctx* c, long long n) {
  if (cluster_form_usable(c)) return run_steps_cluster(c, n);
  TRY(sync_base(c));
  const int G = 64;
  if (n >= G && !c->graph) {
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
    for (int q = 0; q < G; ++q) launch_lattice_step(c->lat, q, true, c->st);
    launch_lattice_advance(c->lat, G, c->st);
    cudaError_t e1 = cudaGetLastError();
    CK(cudaStreamEndCapture(c->st, &g));
    if (e1 != cudaSuccess) {
      cudaGraphDestroy(g);
      return fail(c, VCSGC_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e1));
    }
    cudaError_t e2 = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) return fail(c, VCSGC_ERR_CUDA, std::string("graph: ") + cudaGetErrorString(e2));
    c->graph_steps = G;
  }
  while (n >= G) {
    CK(cudaGraphLaunch(c->graph, c->st));
    c->h_base += G;
    n -= G;
  }
  if (n > 0) {
    for (long long q = 0; q < n; ++q) launch_lattice_step(c->lat, (int)q, true, c->st);
    launch_lattice_advance(c->lat, (int)n, c->st);
    c->h_base += n;
  }
  c->pending = true;
  CK(cudaGetLastError());
  return VCSGC_OK;
}

// apply the pending commit of the last proposed step (fused form); a no-op
// when no step ran since the last flush
int flush(Ctx* c) {
  if (!c->fast || !c->pending) return VCSGC_OK;
  launch_lattice_step(c->lat, 0, false, c->st);
  CK(cudaGetLastError());
  c->pending = false;
  return VCSGC_OK;
}

// refresh the species bytes of replica r (or all when r < 0) from the bits
int sync_bytes(Ctx* c, int r) {
  TRY(sync_from_multi(c));
  if (!c->fast) return VCSGC_OK;
  TRY(flush(c));
  if (r < 0) launch_lattice_unpack(c->lat, c->d_tptr, 0, c->R, c->max_sites, c->st);
  else launch_lattice_unpack(c->lat, c->d_tptr, r, 1, c->h_geom[r].n_sites, c->st);
  CK(cudaGetLastError());
  return VCSGC_OK;
}

int run_steps(Ctx* c, long long n) {
  if (n <= 0) return VCSGC_OK;
  if (c->multi) {
    const int rc = vcsgc_multi_steps(c->multi, n);
    if (rc != VCSGC_OK) return fail(c, rc, vcsgc_multi_last_error(c->multi));
    c->multi_dirty = true;
    return VCSGC_OK;
  }
  if (c->fast) return run_steps_fast(c, n);
  if (c->screen) c->energy_stale = true;
  const int G = 64;
  if (n >= G) {
    if (!c->graph) {
      cudaGraph_t g;
      CK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
      for (int q = 0; q < G; ++q) launch_colour_step(c->mc, c->shell, c->reembed, c->st);
      cudaError_t e1 = cudaGetLastError();
      CK(cudaStreamEndCapture(c->st, &g));
      if (e1 != cudaSuccess) {
        cudaGraphDestroy(g);
        return fail(c, VCSGC_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e1));
      }
      cudaError_t e2 = cudaGraphInstantiate(&c->graph, g, 0);
      cudaGraphDestroy(g);
      if (e2 != cudaSuccess) return fail(c, VCSGC_ERR_CUDA, std::string("graph: ") + cudaGetErrorString(e2));
      c->graph_steps = G;
    }
    while (n >= G) {
      CK(cudaGraphLaunch(c->graph, c->st));
      n -= G;
    }
  }
  for (long long q = 0; q < n; ++q) launch_colour_step(c->mc, c->shell, c->reembed, c->st);
  CK(cudaGetLastError());
  return VCSGC_OK;
}

// species, densities and running state of every replica from the
// multicomponent object after its steps (the energy is recomputed when read)
int sync_from_multi(Ctx* c) {
  if (!c->multi || !c->multi_dirty) return VCSGC_OK;
  for (int r = 0; r < c->R; ++r) {
    MRepState ms;
    const int rc = multi_get_state(c->multi, r, &ms);
    if (rc != VCSGC_OK) return fail(c, rc, vcsgc_multi_last_error(c->multi));
    const uint8_t* t = multi_types_device(c->multi, r);
    if (!t) return fail(c, VCSGC_ERR_CUDA, vcsgc_multi_last_error(c->multi));
    CK(cudaMemcpyAsync(c->rep_types[r], t, c->N, cudaMemcpyDeviceToDevice, c->st));
    TRY(refresh_rho(c, r));
    RepState s;
    std::memset(&s, 0, sizeof(s));
    s.n = ms.cnt[1];
    s.step = ms.step;
    s.fin_step = ms.fin_step;
    s.trials = ms.trials;
    s.local_acc = ms.local_acc;
    s.global_trials = ms.global_trials;
    s.global_acc = ms.global_acc;
    s.flips = ms.flips;
    s.near_ties = ms.near_ties;
    s.steps = ms.steps;
    s.sum_c = ms.sum_c[1];
    s.sum_c2 = ms.sum_c2[1];
    s.s1_acc = ms.s1_acc;
    CK(cudaMemcpyAsync(c->rs + r, &s, sizeof(RepState), cudaMemcpyHostToDevice, c->st));
  }
  CK(cudaStreamSynchronize(c->st));
  c->energy_stale = true;
  c->multi_dirty = false;
  return VCSGC_OK;
}

// this context's species and state of replica r into the multicomponent object
int push_to_multi(Ctx* c, int r, const uint8_t* host_types, const RepState* s) {
  if (!c->multi) return VCSGC_OK;
  int rc = vcsgc_multi_set_types(c->multi, r, host_types);
  if (rc == VCSGC_OK && s) {
    MRepState ms;
    rc = multi_get_state(c->multi, r, &ms);
    ms.step = s->step;
    ms.fin_step = s->fin_step;
    ms.trials = s->trials;
    ms.local_acc = s->local_acc;
    ms.global_trials = s->global_trials;
    ms.global_acc = s->global_acc;
    ms.flips = s->flips;
    ms.near_ties = s->near_ties;
    ms.steps = s->steps;
    ms.s1_acc = s->s1_acc;
    ms.sum_c[1] = s->sum_c;
    ms.sum_c2[1] = s->sum_c2;
    ms.sum_c[0] = (double)s->steps - s->sum_c;
    ms.sum_c2[0] = (double)s->steps - 2.0 * s->sum_c + s->sum_c2;
    if (rc == VCSGC_OK) rc = multi_set_state(c->multi, r, &ms);
  }
  return rc == VCSGC_OK ? VCSGC_OK : fail(c, rc, vcsgc_multi_last_error(c->multi));
}

// ------------------------------------------------------------------- MD
int md_forces(Ctx* c) {
  if (c->d_vir) CK(cudaMemsetAsync(c->d_vir, 0, sizeof(double), c->st));
  launch_md_rho(c->md, c->st);
  launch_md_force(c->md, c->st);
  CK(cudaGetLastError());
  c->forces_valid = true;
  return VCSGC_OK;
}

int md_rebuild(Ctx* c) {
  TRY(build_cell_list(c));
  launch_md_snapshot(c->md, c->st);
  CK(cudaGetLastError());
  return VCSGC_OK;
}

// ----------------------------------------------- Nose-Hoover and MTK (host)
// The extended-system scalars of the MD ensemble (Sec. IV B) are integrated
// here in FP64 with the same Trotter splitting as the per-atom flows the
// kernels apply: Nose-Hoover chains (Martyna, Klein, Tuckerman 1992) on the
// particles and on the barostat, the isotropic MTK barostat (Martyna,
// Tobias, Klein 1994), and the exact sub-flows of Martyna, Tuckerman,
// Tobias, Klein (1996).  N_f = 3 N.
constexpr double BAR_EV_A3 = 6.241509074460763e-07;  // 1 bar in eV / A^3

double sinhc(double x) { return std::fabs(x) < 1e-4 ? 1.0 + x * x / 6.0 + x * x * x * x / 120.0 : std::sinh(x) / x; }

// chain of M links driven by K2 (= sum m v^2 of g degrees of freedom,
// target gkT) for a time h; returns the scale of the coupled velocities
double nhc_step(int M, const double* Q, double* xi, double* eta, double K2, double gkT, double kT, double h) {
  double scale = 1.0;
  for (int pass = 0; pass < 2; ++pass) {
    for (int q = 0; q < M; ++q) {
      const int k = pass == 0 ? M - 1 - q : q;
      const double G = k == 0 ? (K2 * scale * scale - gkT) / Q[0] : (Q[k - 1] * xi[k - 1] * xi[k - 1] - kT) / Q[k];
      const double e = k + 1 < M ? std::exp(-0.25 * h * xi[k + 1]) : 1.0;
      xi[k] = (xi[k] * e + 0.5 * h * G) * e;
    }
    if (pass == 0) {
      scale = std::exp(-h * xi[0]);
      for (int k = 0; k < M; ++k) eta[k] += h * xi[k];
    }
  }
  return scale;
}

// sum of block partials (compensated)
double sum_parts(const std::vector<double>& h) {
  double s = 0.0, c = 0.0;
  for (double v : h) {
    const double t = s + v;
    c += std::fabs(s) >= std::fabs(v) ? (s - t) + v : (v - t) + s;
    s = t;
  }
  return s + c;
}

// sum m v^2 (eV) of replica 0's atoms, with the pending scale applied
int twice_ke_dev(Ctx* c, double* out) {
  const int nb = kinetic_blocks(c->N);
  if (!c->cg_part) TRY(dalloc(c, &c->cg_part, std::max(nb, dot_blocks(3 * c->N))));
  launch_kinetic(c->md, c->cg_part, c->st);
  CK(cudaGetLastError());
  std::vector<double> h(nb);
  CK(cudaMemcpyAsync(h.data(), c->cg_part, sizeof(double) * nb, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  *out = 2.0 * sum_parts(h) * c->nh.vs * c->nh.vs;
  return VCSGC_OK;
}

int read_virial(Ctx* c, double* out) {
  CK(cudaMemcpyAsync(out, c->d_vir, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return VCSGC_OK;
}

void set_box(Ctx* c, double f) {
  for (int q = 0; q < 3; ++q) c->box[q] *= f;
  fill_args(c);
}

// barostat force [alpha K2 + W_vir - 3 V P_ext] / W
double baro_force(const Ctx* c, double K2, double vir) {
  const double nf = 3.0 * (double)c->N, V = c->box[0] * c->box[1] * c->box[2];
  return ((1.0 + 3.0 / nf) * K2 + vir - 3.0 * V * c->nh.p_ext) / c->nh.W;
}

int md_run_nh(Ctx* c, long long n) {
  Ctx::Nh& nh = c->nh;
  const bool npt = nh.kind == 2;
  const double dt = c->dt, h = 0.5 * dt, kT = KB_EV * c->T_md, nf = 3.0 * (double)c->N;
  const double alpha = 1.0 + 3.0 / nf;
  if (!c->forces_valid) TRY(md_forces(c));
  double K2 = 0.0, vir = 0.0;
  TRY(twice_ke_dev(c, &K2));
  TRY(read_virial(c, &vir));
  for (long long q = 0; q < n; ++q) {
    // thermostats, barostat velocity, velocity half kick
    const double s1 = nhc_step(nh.chain, nh.Q, nh.xi, nh.eta, K2, nf * kT, kT, h);
    K2 *= s1 * s1;
    if (npt) {
      nh.veps *= nhc_step(nh.chain, nh.Qb, nh.xib, nh.etab, nh.W * nh.veps * nh.veps, kT, kT, h);
      nh.veps += h * baro_force(c, K2, vir);
    }
    const double a = npt ? alpha * nh.veps : 0.0;
    const double e1 = std::exp(-a * h), he2 = h * std::exp(-0.5 * a * h) * sinhc(0.5 * a * h);
    launch_nh_kick(c->md, nh.vs * s1, e1, he2, c->st);
    nh.vs = 1.0;
    // positions and box
    const double ve = npt ? nh.veps : 0.0;
    const double E1 = std::exp(ve * dt), E2 = dt * std::exp(0.5 * ve * dt) * sinhc(0.5 * ve * dt);
    if (npt) set_box(c, E1);
    CK(cudaMemsetAsync(c->max_disp2, 0, sizeof(unsigned long long), c->st));
    launch_nh_drift(c->md, E1, E2, c->st);
    CK(cudaGetLastError());
    unsigned long long bits = 0;
    CK(cudaMemcpyAsync(&bits, c->max_disp2, sizeof(bits), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    double d2;
    std::memcpy(&d2, &bits, sizeof(d2));
    const double slack = std::fabs(c->md.lam - 1.0) * c->rl;
    if (std::sqrt(d2) + slack > 0.5 * c->skin) {
      TRY(md_rebuild(c));
      fill_args(c);
    }
    TRY(md_forces(c));
    launch_nh_kick(c->md, 1.0, e1, he2, c->st);
    CK(cudaGetLastError());
    TRY(twice_ke_dev(c, &K2));
    if (npt) {
      TRY(read_virial(c, &vir));
      nh.veps += h * baro_force(c, K2, vir);
      nh.veps *= nhc_step(nh.chain, nh.Qb, nh.xib, nh.etab, nh.W * nh.veps * nh.veps, kT, kT, h);
    }
    const double s2 = nhc_step(nh.chain, nh.Q, nh.xi, nh.eta, K2, nf * kT, kT, h);
    K2 *= s2 * s2;
    nh.vs = s2;  // folded into the next kick
    c->md_step++;
  }
  if (nh.vs != 1.0) {
    launch_nh_kick(c->md, nh.vs, 1.0, 0.0, c->st);
    CK(cudaGetLastError());
    nh.vs = 1.0;
  }
  return VCSGC_OK;
}

int md_run(Ctx* c, long long n) {
  if (!c->have_v) return fail(c, VCSGC_ERR_STATE, "md_steps needs velocities (vcsgc_set_velocities)");
  if (c->kind != 1 || c->R != 1) return fail(c, VCSGC_ERR_STATE, "md_steps needs explicit positions and one replica");
  if (c->nh.kind) return md_run_nh(c, n);
  if (!c->forces_valid) TRY(md_forces(c));
  const double half_skin2 = 0.25 * c->skin * c->skin;
  for (long long q = 0; q < n; ++q) {
    launch_md_first_half(c->md, c->md_step, c->st);
    CK(cudaGetLastError());
    unsigned long long bits = 0;
    CK(cudaMemcpyAsync(&bits, c->max_disp2, sizeof(bits), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    double d2;
    std::memcpy(&d2, &bits, sizeof(d2));
    if (d2 > half_skin2) TRY(md_rebuild(c));
    launch_md_rho(c->md, c->st);
    launch_md_force(c->md, c->st);
    launch_md_second_half(c->md, c->st);
    CK(cudaGetLastError());
    c->md_step++;
  }
  return VCSGC_OK;
}

}  // namespace

// =================================================================== C ABI
extern "C" {

int vcsgc_default_options(vcsgc_options* o) {
  if (!o) return VCSGC_ERR_INVALID_ARG;
  std::memset(o, 0, sizeof(*o));
  o->seed = 1;
  o->c0 = -1.0;
  o->kappa_units = 0;
  o->schedule = VCSGC_SCHED_SUBLATTICE;
  o->sched[0] = o->sched[1] = o->sched[2] = 4;
  o->precision = VCSGC_PREC_FP64;
  o->n_replicas = 1;
  o->mass[0] = 55.845;
  o->mass[1] = 63.546;
  o->dt = 2.0;
  o->gamma = 0.01;
  o->T_md = -1.0;
  o->skin = 0.3;
  o->md_seed = 12345;
  o->device = -1;
  return VCSGC_OK;
}

static int setup_fast(Ctx* c, const std::vector<RepState>& hs);
static int cluster_setup(Ctx* c);

static int init_impl(Ctx* c, const vcsgc_lattice* L, const uint8_t* types, const vcsgc_eam_tables* E,
                     double phi, double kappa, double T, const vcsgc_options* o) {
  if (!L || !types || !E || !o) return fail(c, VCSGC_ERR_INVALID_ARG, "null argument");
  if (o->precision != VCSGC_PREC_FP64 && o->precision != VCSGC_PREC_MIXED)
    return fail(c, VCSGC_ERR_INVALID_ARG, "precision must be FP64 or MIXED");
  c->mixed = o->precision == VCSGC_PREC_MIXED;
  if (o->n_replicas < 1) return fail(c, VCSGC_ERR_INVALID_ARG, "n_replicas < 1");
  c->R = o->n_replicas;
  c->kind = L->kind;
  c->rc = E->rc;
  c->skin = L->kind == 1 ? std::max(0.0, o->skin) : 0.0;
  c->rl = c->rc + c->skin;
  if (!(c->rc > 0)) return fail(c, VCSGC_ERR_INVALID_ARG, "rc <= 0");
  if (L->kind == 0) {
    if (L->nx < 1 || L->ny < 1 || L->nz < 1 || !(L->a > 0)) return fail(c, VCSGC_ERR_INVALID_ARG, "bad lattice size");
    c->nx = L->nx; c->ny = L->ny; c->nz = L->nz; c->a = L->a;
    c->N = 2LL * L->nx * L->ny * L->nz;
    c->box[0] = L->a * L->nx; c->box[1] = L->a * L->ny; c->box[2] = L->a * L->nz;
    for (int q = 0; q < 3; ++q)
      if (!(c->box[q] > c->rc)) return fail(c, VCSGC_ERR_INVALID_ARG, "box shorter than r_c (self images)");
  } else if (L->kind == 1) {
    if (L->n < 1 || !L->x || !L->y || !L->z) return fail(c, VCSGC_ERR_INVALID_ARG, "bad explicit lattice");
    c->N = L->n;
    for (int q = 0; q < 3; ++q) {
      c->box[q] = L->box[q];
      if (!(c->box[q] > 2.0 * c->rl) || std::floor(c->box[q] / c->rl) < 3)
        return fail(c, VCSGC_ERR_INVALID_ARG, "box must exceed 2 (r_c + skin) and hold 3 cells");
    }
  } else {
    return fail(c, VCSGC_ERR_INVALID_ARG, "lattice kind must be 0 or 1");
  }
  // the accepted-site list packs a site index and its species in 32 bits
  if (c->N >= (1LL << 30)) return fail(c, VCSGC_ERR_INVALID_ARG, "too many sites (at most 2^30 - 1)");
  if (!(T > 0) || !(kappa >= 0)) return fail(c, VCSGC_ERR_INVALID_ARG, "T must be > 0 and kappa >= 0");
  for (long long i = 0; i < (long long)c->R * c->N; ++i)
    if (types[i] > 1) return fail(c, VCSGC_ERR_INVALID_ARG, "species must be 0 or 1");
  if (E->nr < 2 || E->nrho < 2 || !(E->dr > 0) || !(E->drho > 0))
    return fail(c, VCSGC_ERR_INVALID_ARG, "bad table grid");
  if ((E->nr - 1) * E->dr < c->rc * (1.0 - 1e-12)) return fail(c, VCSGC_ERR_INVALID_ARG, "r table shorter than rc");
  for (int q = 0; q < 3; ++q)
    if (!E->pair[q]) return fail(c, VCSGC_ERR_INVALID_ARG, "missing pair table");
  for (int q = 0; q < 2; ++q)
    if (!E->dens[q] || !E->embed[q]) return fail(c, VCSGC_ERR_INVALID_ARG, "missing table");

  if (o->device >= 0) {
    CK(cudaSetDevice(o->device));
    c->device = o->device;
  } else {
    CK(cudaGetDevice(&c->device));
  }
  if (o->stream) {
    c->st = (cudaStream_t)o->stream;
  } else {
    CK(cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking));
    c->own_stream = true;
  }
  c->mass[0] = o->mass[0] > 0 ? o->mass[0] : 55.845;
  c->mass[1] = o->mass[1] > 0 ? o->mass[1] : 63.546;
  c->dt = o->dt > 0 ? o->dt : 2.0;
  c->gamma = o->gamma >= 0 ? o->gamma : 0.0;
  c->T_md = o->T_md > 0 ? o->T_md : T;
  c->md_seed = o->md_seed;

  // same density function for both species: rho is species-independent and
  // the re-embedding term vanishes identically
  bool same = std::memcmp(E->dens[0], E->dens[1], sizeof(double) * E->nr) == 0;
  if (same) {
    if ((E->ddens[0] == nullptr) != (E->ddens[1] == nullptr)) same = false;
    else if (E->ddens[0] && std::memcmp(E->ddens[0], E->ddens[1], sizeof(double) * E->nr) != 0) same = false;
  }
  c->reembed = !same;
  c->shell = (c->kind == 0);
  if (c->reembed && c->kind == 0)
    for (int q = 0; q < 3; ++q)
      if (!(c->box[q] > 2.0 * c->rc))
        return fail(c, VCSGC_ERR_INVALID_ARG, "species-dependent density needs a box longer than 2 r_c");

  TRY(dalloc(c, &c->derr, 1));
  CK(cudaMemsetAsync(c->derr, 0, sizeof(unsigned), c->st));

  // ---- tables
  for (int q = 0; q < 7; ++q) {
    const bool rgrid = q < 5;
    const int n = rgrid ? E->nr : E->nrho;
    const double h = rgrid ? E->dr : E->drho;
    const double* y = q < 3 ? E->pair[q] : (q < 5 ? E->dens[q - 3] : E->embed[q - 5]);
    const double* m = q < 3 ? E->dpair[q] : (q < 5 ? E->ddens[q - 3] : E->dembed[q - 5]);
    double *dy = nullptr, *dm = nullptr;
    TRY(dalloc(c, &dy, n));
    CK(cudaMemcpyAsync(dy, y, sizeof(double) * n, cudaMemcpyHostToDevice, c->st));
    if (m) {
      TRY(dalloc(c, &dm, n));
      CK(cudaMemcpyAsync(dm, m, sizeof(double) * n, cudaMemcpyHostToDevice, c->st));
    }
    TRY(dalloc(c, &c->coef[q], n - 1));
    launch_spline_coeffs(dy, dm, n, h, c->coef[q], c->st);
    CK(cudaGetLastError());
    Spline& s = c->mc.tab.sp[q];
    s.c = c->coef[q];
    s.inv_h = 1.0 / h;
    s.xmax = (n - 1) * h;
    s.n_int = n - 1;
    TRY(dalloc(c, &c->dcoef[q], n - 1));
    launch_spline_derivs(c->coef[q], n - 1, h, c->dcoef[q], c->st);
    CK(cudaGetLastError());
    Spline& ds = c->mc.tab.dsp[q];
    ds = s;
    ds.c = c->dcoef[q];
    if (c->mixed) {
      Cubic32 *c32 = nullptr, *d32 = nullptr;
      TRY(dalloc(c, &c32, n - 1));
      TRY(dalloc(c, &d32, n - 1));
      launch_to_cubic32(c->coef[q], n - 1, c32, c->st);
      launch_to_cubic32(c->dcoef[q], n - 1, d32, c->st);
      CK(cudaGetLastError());
      Spline32& s32 = c->mc.tab32.sp[q];
      s32.c = c32;
      s32.inv_h = (float)(1.0 / h);
      s32.xmax = (float)((n - 1) * h);
      s32.n_int = n - 1;
      Spline32& ds32 = c->mc.tab32.dsp[q];
      ds32 = s32;
      ds32.c = d32;
    }
  }

  // ---- positions (both kinds; kind 0 from the lattice)
  TRY(dalloc(c, &c->x, c->N));
  TRY(dalloc(c, &c->y, c->N));
  TRY(dalloc(c, &c->z, c->N));
  std::vector<double> hx(c->N), hy(c->N), hz(c->N);
  if (c->kind == 0) {
    for (long long i = 0; i < c->N; ++i) {
      const long long b = i & 1, cell = i >> 1;
      const long long cx = cell % c->nx, cy = (cell / c->nx) % c->ny, cz = cell / ((long long)c->nx * c->ny);
      hx[i] = c->a * (cx + 0.5 * b);
      hy[i] = c->a * (cy + 0.5 * b);
      hz[i] = c->a * (cz + 0.5 * b);
    }
  } else {
    for (long long i = 0; i < c->N; ++i) {
      hx[i] = L->x[i] - c->box[0] * std::floor(L->x[i] / c->box[0]);
      hy[i] = L->y[i] - c->box[1] * std::floor(L->y[i] / c->box[1]);
      hz[i] = L->z[i] - c->box[2] * std::floor(L->z[i] / c->box[2]);
      if (hx[i] >= c->box[0]) hx[i] = 0.0;
      if (hy[i] >= c->box[1]) hy[i] = 0.0;
      if (hz[i] >= c->box[2]) hz[i] = 0.0;
    }
  }
  CK(cudaMemcpyAsync(c->x, hx.data(), sizeof(double) * c->N, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->y, hy.data(), sizeof(double) * c->N, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->z, hz.data(), sizeof(double) * c->N, cudaMemcpyHostToDevice, c->st));
  if (c->mixed) {
    // the mixed form's fixed-point copies, refreshed before each density
    // pass and energy evaluation of the mixed kernels (fix_diff)
    TRY(dalloc(c, &c->ux, c->N));
    TRY(dalloc(c, &c->uy, c->N));
    TRY(dalloc(c, &c->uz, c->N));
    launch_fix_positions(c->N, c->x, c->y, c->z, c->box, c->ux, c->uy, c->uz, c->st);
  }

  // ---- neighbour list (A1)
  TRY(dalloc(c, &c->nbr_cnt, c->N));
  if (c->kind == 0) {
    // BCC half-lattice offsets within r_c, ordered by distance
    struct Off { int h2, x, y, z; };
    std::vector<Off> offs;
    const double ha = 0.5 * c->a;
    const int m = (int)std::ceil(c->rc / ha) + 1;
    for (int x = -m; x <= m; ++x)
      for (int y = -m; y <= m; ++y)
        for (int z = -m; z <= m; ++z) {
          if (((x ^ y) & 1) || ((x ^ z) & 1)) continue;
          const int h2 = x * x + y * y + z * z;
          if (h2 == 0 || ha * ha * h2 >= c->rc * c->rc) continue;
          offs.push_back({h2, x, y, z});
        }
    std::sort(offs.begin(), offs.end(), [](const Off& p, const Off& q) {
      if (p.h2 != q.h2) return p.h2 < q.h2;
      if (p.x != q.x) return p.x < q.x;
      if (p.y != q.y) return p.y < q.y;
      return p.z < q.z;
    });
    if (offs.empty() || (int)offs.size() > MAX_OFFSETS) return fail(c, VCSGC_ERR_INVALID_ARG, "unsupported r_c / a");
    c->K = (int)offs.size();
    std::vector<int3>& h3 = c->offsets;
    std::vector<int> sh2, sz;
    int S = 0;
    for (size_t k = 0; k < offs.size(); ++k) {
      h3.push_back(make_int3(offs[k].x, offs[k].y, offs[k].z));
      if (k == 0 || offs[k].h2 != offs[k - 1].h2) {
        if (S == MAX_SHELLS) return fail(c, VCSGC_ERR_INVALID_ARG, "too many neighbour shells");
        sh2.push_back(offs[k].h2);
        sz.push_back(0);
        ++S;
      }
      sz[S - 1]++;
      c->offset_shell.push_back(S - 1);
      c->mc.shell_end[S - 1] = (int)k + 1;
    }
    c->mc.n_shells = S;
    int3* dh = nullptr;
    int *dh2 = nullptr, *dz = nullptr;
    TRY(dalloc(c, &dh, c->K));
    TRY(dalloc(c, &dh2, S));
    TRY(dalloc(c, &dz, S));
    CK(cudaMemcpyAsync(dh, h3.data(), sizeof(int3) * c->K, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(dh2, sh2.data(), sizeof(int) * S, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(dz, sz.data(), sizeof(int) * S, cudaMemcpyHostToDevice, c->st));
    TRY(dalloc(c, &c->nbr, (size_t)c->N * c->K));
    launch_lattice_neighbours(c->nx, c->ny, c->nz, dh, c->K, c->nbr, c->nbr_cnt, c->st);
    TRY(dalloc(c, &c->shell_tab, 1 + 3 * S));
    launch_shell_tables(c->mc.tab, dh2, dz, S, c->a, c->shell_tab, c->derr, c->st,
                        c->mixed ? &c->mc.tab32 : nullptr);
    CK(cudaGetLastError());
  } else {
    const double dens = c->N / (c->box[0] * c->box[1] * c->box[2]);
    const double est = 4.0 / 3.0 * M_PI * c->rl * c->rl * c->rl * dens;
    c->K = ((int)(est * 1.4) + 16 + 7) / 8 * 8;
    TRY(dalloc(c, &c->nbr, (size_t)c->N * c->K));
    c->mc.n_shells = 0;
    TRY(dalloc(c, &c->shell_tab, 1));
  }
  // ---- buffers
  TRY(dalloc(c, &c->types, (size_t)c->R * c->N));
  CK(cudaMemcpyAsync(c->types, types, (size_t)c->R * c->N, cudaMemcpyHostToDevice, c->st));
  c->rep_types.resize(c->R);
  c->rep_n.assign(c->R, c->N);
  for (int r = 0; r < c->R; ++r) c->rep_types[r] = c->types + (long long)r * c->N;
  TRY(dalloc(c, &c->rho, (size_t)(c->reembed ? c->R : 1) * c->N));
  TRY(dalloc(c, &c->dF, c->N));
  TRY(dalloc(c, &c->dFp, c->N));
  TRY(dalloc(c, &c->dFp32, c->N));
  TRY(dalloc(c, &c->fx, c->N));
  TRY(dalloc(c, &c->fy, c->N));
  TRY(dalloc(c, &c->fz, c->N));
  TRY(dalloc(c, &c->x0, c->N));
  TRY(dalloc(c, &c->y0, c->N));
  TRY(dalloc(c, &c->z0, c->N));
  TRY(dalloc(c, &c->max_disp2, 1));
  TRY(dalloc(c, &c->d_vir, 1));
  TRY(dalloc(c, &c->rp, c->R));
  TRY(dalloc(c, &c->rs, c->R));
  TRY(dalloc(c, &c->acc, c->R));
  CK(cudaMemsetAsync(c->rs, 0, sizeof(RepState) * c->R, c->st));
  CK(cudaMemsetAsync(c->acc, 0, sizeof(StepAcc) * c->R, c->st));
  c->part_n = std::max(energy_blocks(c->N), kinetic_blocks(c->N));
  TRY(dalloc(c, &c->part, c->part_n));
  fill_args(c);
  if (c->kind == 1) TRY(md_rebuild(c));

  // ---- schedule (A3)
  c->sched_kind = o->schedule;
  std::memcpy(c->sched, o->sched, sizeof(c->sched));
  {
    Sched S;
    TRY(build_schedule(c, hx, hy, hz, S));
    TRY(upload_schedule(c, S));
  }

  // ---- replica parameters (Eq. pi_vcsgc, Eq. trans_vcsgc_par1)
  c->h_rp.resize(c->R);
  std::vector<RepState> hs(c->R);
  std::memset(hs.data(), 0, sizeof(RepState) * c->R);
  for (int r = 0; r < c->R; ++r) {
    const double ph = o->phi_r ? o->phi_r[r] : phi;
    const double ka = o->kappa_r ? o->kappa_r[r] : kappa;
    const double TT = o->T_r ? o->T_r[r] : T;
    const uint64_t seed = o->seed_r ? o->seed_r[r] : o->seed + (uint64_t)r;
    const double c0r = o->c0_r ? o->c0_r[r] : o->c0;
    if (!(TT > 0) || !(ka >= 0)) return fail(c, VCSGC_ERR_INVALID_ARG, "replica T must be > 0, kappa >= 0");
    long long nb = 0;
    for (long long i = 0; i < c->N; ++i) nb += types[(long long)r * c->N + i];
    RepParams& p = c->h_rp[r];
    p.beta = 1.0 / (KB_EV * TT);
    p.kappa_p = o->kappa_units == 1 ? ka : ka * KB_EV * TT / (double)c->N;
    const double c0 = c0r < 0 ? (double)nb / (double)c->N : c0r;
    p.n0 = (double)c->N * c0;
    p.dmu0 = ph + 2.0 * p.kappa_p * p.n0;
    p.phi = ph;
    p.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    hs[r].n = nb;
  }
  CK(cudaMemcpyAsync(c->rp, c->h_rp.data(), sizeof(RepParams) * c->R, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->rs, hs.data(), sizeof(RepState) * c->R, cudaMemcpyHostToDevice, c->st));

  // ---- screened re-embedding on the rigid lattice
  if (c->kind == 0 && c->reembed && c->shell && c->mc.n_shells > 0) TRY(screen_setup(c));
  // ---- rho, dF and energies (A2)
  if (c->reembed) {
    for (int r = 0; r < c->R; ++r) TRY(refresh_rho(c, r));
  } else {
    TRY(refresh_rho(c, 0));
  }
  TRY(check_device_error(c));
  for (int r = 0; r < c->R; ++r) {
    double e;
    TRY(energy_of(c, r, &e));
    CK(cudaMemcpyAsync(&c->rs[r].energy, &e, sizeof(double), cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
  }
  if (c->kind == 1 && c->R == 1) TRY(md_forces(c));
  TRY(check_device_error(c));
  TRY(setup_fast(c, hs));
  // species-dependent densities on the period-q sublattice with the
  // five-shell table: the colour steps run through a two-species
  // multicomponent object, whose FP32-screened kernels (compile-time
  // offsets, per-site floats ordered by x mod period) advance the same chain
  // step for step
  if (c->kind == 0 && c->reembed && c->sched_kind == VCSGC_SCHED_SUBLATTICE && o->kappa_units == 0 && !c->mixed &&
      !c->no_fast && c->mc.n_shells == 5 && c->K == 58) {
    vcsgc_multi_tables mt{};
    mt.K = 2;
    mt.nr = E->nr;
    mt.dr = E->dr;
    mt.nrho = E->nrho;
    mt.drho = E->drho;
    mt.rc = E->rc;
    for (int q = 0; q < 3; ++q) {
      mt.pair[q] = E->pair[q];  // (0,0), (0,1), (1,1)
      mt.dpair[q] = E->dpair[q];
    }
    for (int q = 0; q < 2; ++q) {
      mt.dens[q] = E->dens[q];
      mt.ddens[q] = E->ddens[q];
      mt.embed[q] = E->embed[q];
      mt.dembed[q] = E->dembed[q];
    }
    std::vector<double> ph(c->R), ka(c->R), TT(c->R), cc(c->R);
    std::vector<uint64_t> sd(c->R);
    for (int r = 0; r < c->R; ++r) {
      ph[r] = o->phi_r ? o->phi_r[r] : phi;
      ka[r] = o->kappa_r ? o->kappa_r[r] : kappa;
      TT[r] = o->T_r ? o->T_r[r] : T;
      cc[r] = o->c0_r ? o->c0_r[r] : o->c0;
      sd[r] = o->seed_r ? o->seed_r[r] : o->seed + (uint64_t)r;
    }
    const int32_t period[3] = {c->sched[0], c->sched[1], c->sched[2]};
    void* m = nullptr;
    const int rc = vcsgc_multi_init(&m, L, types, &mt, c->R, ph.data(), ka.data(), TT.data(), cc.data(), sd.data(),
                                    period, c->st, c->device);
    if (rc != VCSGC_OK) return fail(c, rc, std::string("multicomponent engine: ") + vcsgc_multi_last_error(nullptr));
    if (multi_screened(m)) {
      c->multi = m;
    } else {
      vcsgc_multi_free(m);
    }
  }
  return VCSGC_OK;
}

// Shared part of the fused bit-packed form (rows and shell masks of the
// neighbourhood, shell constants, dF): 0 when set up, 1 when the lattice is
// outside the form (the two-launch colour step is used instead).
static int lattice_shared(Ctx* c, int& unsupported) {
  unsupported = 1;
  if (c->kind != 0 || c->reembed || c->nx < 2) return VCSGC_OK;
  // index arithmetic of the fused form: sites < 2^22, rows < 2^20, 2 nx < 2048
  if (c->N > (1LL << 22) || 2 * c->nx >= 2048 || (long long)c->ny * c->nz >= (1LL << 20)) return VCSGC_OK;
  if (c->sched_kind != VCSGC_SCHED_BLOCKS && c->sched_kind != VCSGC_SCHED_SUBLATTICE &&
      c->sched_kind != VCSGC_SCHED_OVERLAP)
    return VCSGC_OK;
  const int S = c->mc.n_shells;
  if (S > LAT_MAX_SH) return VCSGC_OK;
  LatArgs& l = c->lat;
  int hmax = 0;
  for (const int3& h : c->offsets) hmax = std::max(hmax, std::abs(h.x));
  if (hmax > LAT_HALO) return VCSGC_OK;
  for (int b = 0; b < 2; ++b) {
    int nr = 0;
    for (size_t k = 0; k < c->offsets.size(); ++k) {
      const int3 h = c->offsets[k];
      // neighbour row: floor((2Y + b + hy) / 2) - Y
      const int dy = (int)std::floor((b + h.y) / 2.0), dz = (int)std::floor((b + h.z) / 2.0);
      int q = 0;
      while (q < nr && (l.rows[b][q].dy != dy || l.rows[b][q].dz != dz)) ++q;
      if (q == nr) {
        if (nr == LAT_MAX_ROWS) return VCSGC_OK;
        l.rows[b][q].dy = dy;
        l.rows[b][q].dz = dz;
        for (int s = 0; s < LAT_MAX_SH; ++s) l.rows[b][q].mask[s] = 0u;
        ++nr;
      }
      l.rows[b][q].mask[c->offset_shell[k]] |= 1u << (h.x + hmax);
    }
    l.n_rows[b] = nr;
  }
  std::vector<double> tab(1 + 3 * S);
  CK(cudaMemcpyAsync(tab.data(), c->shell_tab, sizeof(double) * tab.size(), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  l.C = tab[0];
  for (int s = 0; s < LAT_MAX_SH; ++s) {
    l.G[s] = s < S ? tab[1 + s] : 0.0;
    l.G32[s] = (float)l.G[s];
  }
  // dF_i = F_B(rho_i) - F_A(rho_i): uniform on a perfect lattice
  std::vector<double> dF(c->N);
  CK(cudaMemcpyAsync(dF.data(), c->dF, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  bool uni = true;
  c->df_absmax = 0.0;
  for (long long i = 0; i < c->N; ++i) {
    if (dF[i] != dF[0]) uni = false;
    c->df_absmax = std::max(c->df_absmax, std::fabs(dF[i]));
  }
  l.df_uniform = uni ? 1 : 0;
  l.dF0 = dF[0];
  float* df32 = nullptr;
  TRY(dalloc(c, &df32, c->N));
  launch_to_float(c->dF, df32, c->N, c->st);
  CK(cudaGetLastError());
  l.dF = c->dF;
  l.dF32 = df32;
  l.hmax = hmax;
  l.n_shells = S;
  l.bcc5 = lattice_rows_bcc5(l) ? 1 : 0;
  std::vector<int> zs(S, 0);
  for (int sh : c->offset_shell) zs[sh]++;
  c->sum_absG = 0.0;
  for (int s = 0; s < S; ++s) c->sum_absG += zs[s] * std::fabs(l.G[s]);
  if (uni) {
    // energy of a species array set from the host: shell pair values and
    // F_A, F_B at the uniform density
    LatZ z{};
    for (int s = 0; s < S; ++s) z.z[s] = zs[s];
    TRY(dalloc(c, &c->etab, 4 * S + 2));
    launch_lattice_energy_table(c->mc.tab, c->mixed ? &c->mc.tab32 : nullptr, c->shell_tab, S, z, c->rho,
                                c->etab, c->derr, c->st);
    CK(cudaGetLastError());
  }
  unsupported = 0;
  return VCSGC_OK;
}

// FP32-screen constants of replica parameters p (bound on |X32 - X|)
static LatRep lattice_rep(const Ctx* c, const RepParams& p) {
  const LatArgs& l = c->lat;
  const int S = l.n_shells;
  LatRep lr;
  const double cpd = l.C + p.dmu0 + (l.df_uniform ? l.dF0 : 0.0);
  const double M = std::fabs(l.C) + std::fabs(p.dmu0) + c->sum_absG + c->df_absmax + std::fabs(cpd);
  lr.cpd32 = (float)cpd;
  lr.beta32 = (float)p.beta;
  // (2 S + 3) roundings of at most 2^-24 M each, times beta, four-fold margin
  lr.dx = (float)(4.0 * p.beta * (2 * S + 3) * std::ldexp(M, -24));
  lr.bk32 = (float)(p.beta * p.kappa_p);
  lr.n0_32 = (float)p.n0;
  lr.pad[0] = lr.pad[1] = lr.pad[2] = 0.0f;
  return lr;
}

static LatGeom lattice_geom(int nx, int ny, int nz, const int q[3], int d, int dmax, long long bits_off,
                            long long pend_off) {
  LatGeom g;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.W = (2 * nx + 2 * LAT_HALO + 31) / 32;
  g.bits_off = bits_off;
  g.pend_off = pend_off;
  g.n_sites = 2LL * nx * ny * nz;
  g.d = d;
  g.dmax = dmax;
  g.rcp_nx = 1.0f / (float)nx;
  g.rcp_ny = 1.0f / (float)ny;
  g.nxq = q ? nx / q[0] : 0;
  g.nyq = q ? ny / q[1] : 0;
  g.rcp_nxq = q ? 1.0f / (float)g.nxq : 0.0f;
  g.rcp_nyq = q ? 1.0f / (float)g.nyq : 0.0f;
  return g;
}

// Allocate and initialise the per-replica state of the fused form: rows of
// all replicas in one array, accumulators, pending slots; pack the species.
static int lattice_state(Ctx* c, const std::vector<long long>& n0, const std::vector<LatRep>& lr) {
  LatArgs& l = c->lat;
  const int R = c->R;
  long long words = 0, slots = 0;
  int dmax = 0;
  for (const LatGeom& g : c->h_geom) {
    words = std::max(words, g.bits_off + (long long)g.ny * g.nz * g.W);
    slots = std::max(slots, g.pend_off + g.dmax);
    dmax = std::max(dmax, g.dmax);
  }
  LatGeom* dg = nullptr;
  LatRep* dlr = nullptr;
  TRY(dalloc(c, &dg, R));
  TRY(dalloc(c, &dlr, R));
  TRY(dalloc(c, &l.bits, (size_t)(words + 1)));
  TRY(dalloc(c, &l.acc, (size_t)R * 3));
  TRY(dalloc(c, &l.n_start, (size_t)R * 2));
  TRY(dalloc(c, &l.pend, (size_t)slots));
  TRY(dalloc(c, &l.ctl, 1));
  TRY(dalloc(c, &l.ctab, (size_t)R * LAT_CTAB));
  TRY(dalloc(c, &l.ugtab, (size_t)R * LAT_CTAB));
  c->max_words = c->max_sites = 0;
  for (const LatGeom& g : c->h_geom) {
    c->max_words = std::max(c->max_words, (long long)g.ny * g.nz * g.W);
    c->max_sites = std::max(c->max_sites, g.n_sites);
  }
  c->epstride = lattice_energy_blocks(c->max_words);
  TRY(dalloc(c, &c->epart, (size_t)((long long)lattice_energy_width() * R * c->epstride)));
  TRY(dalloc(c, &c->d_tptr, (size_t)R));
  CK(cudaMemcpyAsync(c->d_tptr, c->rep_types.data(), sizeof(uint8_t*) * R, cudaMemcpyHostToDevice, c->st));
  // four sites per thread in the unpack: every replica's rows of even length
  // and species bytes starting 4-byte aligned
  l.unpack4 = 1;
  for (int r = 0; r < R; ++r)
    if ((c->h_geom[r].nx & 1) || ((uintptr_t)c->rep_types[r] & 3)) l.unpack4 = 0;
  CK(cudaMemcpyAsync(dg, c->h_geom.data(), sizeof(LatGeom) * R, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(dlr, lr.data(), sizeof(LatRep) * R, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemsetAsync(l.bits, 0, sizeof(unsigned long long) * (words + 1), c->st));
  CK(cudaMemsetAsync(l.acc, 0, sizeof(StepAcc) * R * 3, c->st));
  CK(cudaMemsetAsync(l.pend, 0xFF, sizeof(int) * slots, c->st));
  CK(cudaMemsetAsync(l.ctl, 0, sizeof(LatCtl), c->st));
  std::vector<long long> ns(2 * R, 0);
  for (int r = 0; r < R; ++r) ns[2 * r] = n0[r];
  CK(cudaMemcpyAsync(l.n_start, ns.data(), sizeof(long long) * ns.size(), cudaMemcpyHostToDevice, c->st));
  // fin_step = -1: no step finalised yet
  std::vector<RepState> rs(R);
  CK(cudaMemcpyAsync(rs.data(), c->rs, sizeof(RepState) * R, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  for (auto& st : rs) st.fin_step = -1;
  CK(cudaMemcpyAsync(c->rs, rs.data(), sizeof(RepState) * R, cudaMemcpyHostToDevice, c->st));
  // block tables: each replica gets ceil(dmax_r / BS) blocks (at least one,
  // whose first thread-warp finalises the replica's steps)
  const int bsz[3] = {64, 128, 256};
  for (int q = 0; q < 3; ++q) {
    std::vector<int2> tab;
    for (int r = 0; r < R; ++r) {
      const int nb = std::max(1, (c->h_geom[r].dmax + bsz[q] - 1) / bsz[q]);
      for (int b = 0; b < nb; ++b) tab.push_back(make_int2(r, b * bsz[q]));
    }
    TRY(dalloc(c, &c->blk_tab[q], tab.size()));
    CK(cudaMemcpyAsync(c->blk_tab[q], tab.data(), sizeof(int2) * tab.size(), cudaMemcpyHostToDevice, c->st));
    c->n_blk_tab[q] = (int)tab.size();
  }
  l.geom = dg;
  l.lrep = dlr;
  l.dmax = dmax;
  l.R = R;
  if (l.block == 0) {
    l.block = 128;
    // prefetching helps while one launch fits in one wave of resident blocks
    // (4 per SM at its register count); past that, occupancy matters more
    long long trials = 0;
    for (const LatGeom& g : c->h_geom) trials += g.dmax;
    l.prefetch = trials <= 152LL * 4 * 128 ? 1 : 0;
  }
  select_blk(c);
  c->fast = true;
  fill_args(c);
  launch_lattice_pack(l, c->d_tptr, 0, R, c->max_words, c->st);
  launch_colour_table(l, c->st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->st));
  c->h_base = 0;
  c->pending = false;
  drop_graph(c);
  TRY(cluster_setup(c));
  return check_device_error(c);
}

// Tilings of the cluster-resident form.  For each cluster size s in 1, 2,
// 4, 8, 16 every replica needs a TY x TZ = s grid of tiles dividing its
// ny x nz rows with Ty, Tz >= 2, whose rows with halo, (Ty + 4)(Tz + 4) W
// words, and accept lists fit in shared memory, and whose trials per step
// fit the threads; among such grids the one with whole sublattice periods
// per tile (equal trials per CTA) and the squarest tile is taken.  Sizes
// the GPU cannot co-schedule (cudaOccupancyMaxActiveClusters = 0) are
// dropped.
static int cluster_setup(Ctx* c) {
  const LatArgs& l = c->lat;
  if (!l.sublattice || !l.bcc5 || !l.df_uniform || l.n_shells != 5) return VCSGC_OK;
  const int sizes[5] = {1, 2, 4, 8, 16};
  for (int qi = 0; qi < 5; ++qi) {
    const int s = sizes[qi];
    std::vector<ClTile> tiles;
    size_t smem = 0;
    bool ok = true;
    for (int r = 0; r < c->R && ok; ++r) {
      const LatGeom& g = c->h_geom[r];
      ClTile best{};
      bool found = false;
      long long best_score = 0;
      for (int TY = 1; TY <= s; TY *= 2) {
        const int TZ = s / TY;
        if (g.ny % TY || g.nz % TZ) continue;
        const int Ty = g.ny / TY, Tz = g.nz / TZ;
        if (Ty < 2 || Tz < 2) continue;
        ClTile t{TY, TZ, Ty, Tz, 0};
        t.lcap = ((Ty + l.qy - 1) / l.qy) * ((Tz + l.qz - 1) / l.qz) * g.nxq;
        if (t.lcap > 512 * CL_TRIALS_PER_THREAD) continue;
        const size_t sm = cluster_smem_bytes(t, g.W);
        if (sm > CL_SMEM_MAX) continue;
        const bool whole = Ty % l.qy == 0 && Tz % l.qz == 0;
        const long long score = (whole ? 1LL << 40 : 0) - (long long)std::abs(Ty - Tz);
        if (!found || score > best_score) {
          found = true;
          best_score = score;
          best = t;
        }
      }
      if (!found) ok = false;
      tiles.push_back(best);
      smem = std::max(smem, cluster_smem_bytes(best, g.W));
      c->cl_lcap[qi] = std::max(c->cl_lcap[qi], best.lcap);
    }
    if (!ok || cluster_capacity(s, 512, smem) < 1) continue;
    TRY(dalloc(c, &c->cl_tiles[qi], tiles.size()));
    CK(cudaMemcpyAsync(c->cl_tiles[qi], tiles.data(), sizeof(ClTile) * tiles.size(), cudaMemcpyHostToDevice, c->st));
    c->cl_smem[qi] = smem;
  }
  return VCSGC_OK;
}

// The fused bit-packed form applies to a rigid lattice with one density
// function and a BLOCKS or SUBLATTICE schedule.
static int setup_fast(Ctx* c, const std::vector<RepState>& hs) {
  if (c->no_fast) return VCSGC_OK;
  int unsupported = 1;
  TRY(lattice_shared(c, unsupported));
  if (unsupported) return VCSGC_OK;
  LatArgs& l = c->lat;
  const int q[3] = {c->sched[0], c->sched[1], c->sched[2]};
  const bool sub = c->sched_kind == VCSGC_SCHED_SUBLATTICE;
  if (sub) {
    l.rcp_qx = 1.0f / (float)q[0];
    l.rcp_qy = 1.0f / (float)q[1];
  }
  c->h_geom.clear();
  const long long W = (2 * c->nx + 2 * LAT_HALO + 31) / 32;
  for (int r = 0; r < c->R; ++r) {
    c->h_geom.push_back(lattice_geom(c->nx, c->ny, c->nz, sub ? q : nullptr, c->sublattice_d, c->dmax,
                                     (long long)r * c->ny * c->nz * W, (long long)r * c->dmax));
    c->h_geom.back().site_off = (long long)r * c->N;
  }
  std::vector<long long> n0(c->R);
  std::vector<LatRep> lr(c->R);
  for (int r = 0; r < c->R; ++r) {
    n0[r] = hs[r].n;
    lr[r] = lattice_rep(c, c->h_rp[r]);
  }
  return lattice_state(c, n0, lr);
}

static void destroy(Ctx* c) {
  if (!c) return;
  if (c->multi) vcsgc_multi_free(c->multi);
  c->multi = nullptr;
  for (Ctx* sc : c->subs) destroy(sc);
  c->subs.clear();
  drop_graph(c);
  if (c->st) cudaStreamSynchronize(c->st);
  if (c->h_pin) cudaFreeHost(c->h_pin);
  for (void* p : c->allocs) cudaFree(p);
  if (c->own_stream && c->st) cudaStreamDestroy(c->st);
  delete c;
}

int vcsgc_init(void** out, const vcsgc_lattice* L, const uint8_t* types, const vcsgc_eam_tables* E,
               double phi, double kappa, double T, const vcsgc_options* opt) {
  VCSGC_TRACE("vcsgc_init");
  if (!out) return VCSGC_ERR_INVALID_ARG;
  *out = nullptr;
  vcsgc_options def;
  vcsgc_default_options(&def);
  Ctx* c = new (std::nothrow) Ctx();
  if (!c) {
    g_init_error = "host allocation failed";
    return VCSGC_ERR_NOMEM;
  }
  const int rc = init_impl(c, L, types, E, phi, kappa, T, opt ? opt : &def);
  if (rc != VCSGC_OK) {
    g_init_error = c->err;
    destroy(c);
    return rc;
  }
  *out = c;
  return VCSGC_OK;
}

void vcsgc_free(void* ctx) { destroy(static_cast<Ctx*>(ctx)); }

// Batch of rigid BCC lattices of different sizes: each replica is set up by a
// context of its own (neighbour list, rho, energy, shell constants), then all
// replicas' species are packed into one bit array and advanced by the same
// fused colour-step launches.
static int batch_impl(Ctx* c, int32_t n_rep, const int32_t* cells, double a, const uint8_t* types,
                      const vcsgc_eam_tables* E, const double* phi, const double* kappa, const double* T,
                      const vcsgc_options* o) {
  if (n_rep < 1 || !cells || !types || !E || !phi || !kappa || !T || !o)
    return fail(c, VCSGC_ERR_INVALID_ARG, "null argument or no replicas");
  if (o->schedule != VCSGC_SCHED_SUBLATTICE) return fail(c, VCSGC_ERR_INVALID_ARG, "a batch needs the SUBLATTICE schedule");
  if (o->device >= 0) {
    CK(cudaSetDevice(o->device));
    c->device = o->device;
  } else {
    CK(cudaGetDevice(&c->device));
  }
  if (o->stream) {
    c->st = (cudaStream_t)o->stream;
  } else {
    CK(cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking));
    c->own_stream = true;
  }
  c->R = n_rep;
  c->kind = 0;
  c->sched_kind = o->schedule;
  std::memcpy(c->sched, o->sched, sizeof(c->sched));
  c->mixed = o->precision == VCSGC_PREC_MIXED;
  long long off = 0;
  for (int r = 0; r < n_rep; ++r) {
    vcsgc_options so = *o;
    so.n_replicas = 1;
    so.phi_r = so.kappa_r = so.T_r = so.c0_r = nullptr;
    so.seed_r = nullptr;
    so.seed = o->seed_r ? o->seed_r[r] : o->seed + (uint64_t)r;
    so.c0 = o->c0_r ? o->c0_r[r] : o->c0;
    so.stream = c->st;
    vcsgc_lattice L;
    std::memset(&L, 0, sizeof(L));
    L.kind = 0;
    L.nx = cells[3 * r];
    L.ny = cells[3 * r + 1];
    L.nz = cells[3 * r + 2];
    L.a = a;
    Ctx* sc = new (std::nothrow) Ctx();
    if (!sc) return fail(c, VCSGC_ERR_NOMEM, "host allocation failed");
    sc->no_fast = true;
    c->subs.push_back(sc);
    const int rc = init_impl(sc, &L, types + off, E, phi[r], kappa[r], T[r], &so);
    if (rc != VCSGC_OK) return fail(c, rc, "replica " + std::to_string(r) + ": " + sc->err);
    off += sc->N;
  }
  Ctx* s0 = c->subs[0];
  // shared parts from the first replica; every replica shares a, r_c and
  // the tables, hence the neighbourhood and the shell constants
  c->nx = s0->nx; c->ny = s0->ny; c->nz = s0->nz; c->a = a;
  c->N = s0->N;
  c->dF = s0->dF;
  c->rho = s0->rho;
  c->mc.tab = s0->mc.tab;
  c->mc.tab32 = s0->mc.tab32;
  c->shell_tab = s0->shell_tab;
  c->mc.n_shells = s0->mc.n_shells;
  c->offsets = s0->offsets;
  c->offset_shell = s0->offset_shell;
  c->n_colours = s0->n_colours;
  c->col_start = s0->col_start;
  c->dom_start = s0->dom_start;
  c->dom_sites = s0->dom_sites;
  c->steps_per_sweep = s0->steps_per_sweep;
  TRY(dalloc(c, &c->derr, 1));
  CK(cudaMemsetAsync(c->derr, 0, sizeof(unsigned), c->st));
  int unsupported = 1;
  TRY(lattice_shared(c, unsupported));
  if (unsupported || !c->lat.df_uniform)
    return fail(c, VCSGC_ERR_INVALID_ARG, "a batch needs perfect rigid lattices with one density function");
  const int q[3] = {c->sched[0], c->sched[1], c->sched[2]};
  c->lat.rcp_qx = 1.0f / (float)q[0];
  c->lat.rcp_qy = 1.0f / (float)q[1];
  c->h_geom.clear();
  c->rep_types.clear();
  c->rep_n.clear();
  c->h_rp.clear();
  std::vector<long long> n0;
  std::vector<LatRep> lr;
  std::vector<RepState> rs;
  long long words = 0, slots = 0, sites = 0;
  for (int r = 0; r < n_rep; ++r) {
    Ctx* sc = c->subs[r];
    if (sc->steps_per_sweep != c->steps_per_sweep || sc->mc.n_shells != c->mc.n_shells)
      return fail(c, VCSGC_ERR_INVALID_ARG, "replicas must share the schedule period");
    LatGeom g = lattice_geom(sc->nx, sc->ny, sc->nz, q, sc->sublattice_d, sc->dmax, words, slots);
    g.site_off = sites;
    sites += g.n_sites;
    words += (long long)g.ny * g.nz * g.W;
    slots += g.dmax;
    c->h_geom.push_back(g);
    c->rep_types.push_back(sc->types);
    c->rep_n.push_back(sc->N);
    c->h_rp.push_back(sc->h_rp[0]);
    RepState st;
    CK(cudaMemcpyAsync(&st, sc->rs, sizeof(RepState), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    n0.push_back(st.n);
    rs.push_back(st);
    lr.push_back(lattice_rep(c, sc->h_rp[0]));
  }
  c->dmax = 0;
  for (const LatGeom& g : c->h_geom) c->dmax = std::max(c->dmax, g.dmax);
  TRY(dalloc(c, &c->rp, n_rep));
  TRY(dalloc(c, &c->rs, n_rep));
  CK(cudaMemcpyAsync(c->rp, c->h_rp.data(), sizeof(RepParams) * n_rep, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->rs, rs.data(), sizeof(RepState) * n_rep, cudaMemcpyHostToDevice, c->st));
  c->sublattice_d = s0->sublattice_d;
  return lattice_state(c, n0, lr);
}

int vcsgc_batch_init(void** out, int32_t n_rep, const int32_t* cells, double a, const uint8_t* types,
                     const vcsgc_eam_tables* E, const double* phi, const double* kappa, const double* T,
                     const vcsgc_options* opt) {
  VCSGC_TRACE("vcsgc_batch_init");
  if (!out) return VCSGC_ERR_INVALID_ARG;
  *out = nullptr;
  vcsgc_options def;
  vcsgc_default_options(&def);
  Ctx* c = new (std::nothrow) Ctx();
  if (!c) {
    g_init_error = "host allocation failed";
    return VCSGC_ERR_NOMEM;
  }
  const int rc = batch_impl(c, n_rep, cells, a, types, E, phi, kappa, T, opt ? opt : &def);
  if (rc != VCSGC_OK) {
    g_init_error = c->err;
    destroy(c);
    return rc;
  }
  *out = c;
  return VCSGC_OK;
}

int vcsgc_autotune(void* ctx, int64_t steps, int32_t* best_block) {
  VCSGC_TRACE("vcsgc_autotune");
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || steps < 1 || !best_block) return VCSGC_ERR_INVALID_ARG;
  if (!c->fast) {
    *best_block = MC_BLOCK;
    return VCSGC_OK;
  }
  // candidates (form, block, variant): one launch per colour step with block
  // size x row prefetch (prefetching shortens the dependent chain of a step
  // but costs registers, i.e. resident blocks), then the cluster-resident
  // form with each cluster size that serves these lattices x block size
  std::vector<std::array<int, 3>> cand = {{0, 64, 1}, {0, 128, 1}, {0, 256, 1}, {0, 64, 0}, {0, 128, 0}, {0, 256, 0}};
  if (!c->lat.da)
    for (int s : {1, 2, 4, 8, 16})
      if (c->cl_tiles[cl_index(s)])
        for (int b : {256, 512}) cand.push_back({1, b, s});
  float best = 0.0f;
  std::array<int, 3> bc = {0, 128, 1};
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (const auto& cb : cand) {
    if (vcsgc_set_launch(c, cb[0], cb[1], cb[2]) != VCSGC_OK) continue;
    // one untimed step with the candidate, then the timed ones
    TRY(run_steps_fast(c, 1));
    CK(cudaEventRecord(e0, c->st));
    TRY(run_steps_fast(c, steps));
    CK(cudaEventRecord(e1, c->st));
    CK(cudaEventSynchronize(e1));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (best == 0.0f || ms < best) {
      best = ms;
      bc = cb;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->err.clear();
  TRY(vcsgc_set_launch(c, bc[0], bc[1], bc[2]));
  *best_block = bc[1];
  return check_device_error(c);
}

// A new colour schedule for a rigid-lattice context, mid-chain.  Every
// schedule leaves pi_V invariant (its composite moves satisfy detailed
// balance on their own), so a chain may change schedules between colour
// steps; the step counter, and with it the random streams, runs on.  The
// fused form's per-schedule data (domains per colour, pending slots, block
// tables, colour table, cluster tilings) is rebuilt; species, running state
// and step base are kept.
static int reschedule(Ctx* c, int kind, const int32_t sched[6]) {
  if (c->kind != 0 || !c->subs.empty() || c->multi || c->no_fast)
    return fail(c, VCSGC_ERR_STATE, "schedule change: rigid single-lattice contexts only");
  if (kind != VCSGC_SCHED_BLOCKS && kind != VCSGC_SCHED_SUBLATTICE && kind != VCSGC_SCHED_OVERLAP)
    return fail(c, VCSGC_ERR_INVALID_ARG, "schedule change: BLOCKS, SUBLATTICE or OVERLAP");
  TRY(sync_bytes(c, -1));  // the pending step committed, the species bytes current
  const int old_kind = c->sched_kind;
  int old_sched[6];
  std::memcpy(old_sched, c->sched, sizeof(old_sched));
  c->sched_kind = kind;
  std::memcpy(c->sched, sched, sizeof(c->sched));
  Sched S;
  const std::vector<double> none;
  const int rc = build_schedule(c, none, none, none, S);
  if (rc != VCSGC_OK) {
    c->sched_kind = old_kind;
    std::memcpy(c->sched, old_sched, sizeof(old_sched));
    return rc;
  }
  int dnew = 0;  // domains of the fullest colour: the fused form's trials per replica and step
  for (size_t k = 0; k + 1 < S.col.size(); ++k) dnew = std::max(dnew, S.col[k + 1] - S.col[k]);
  TRY(upload_schedule(c, S));
  drop_graph(c);
  if (!c->fast) return check_device_error(c);
  c->dmax = dnew;
  LatArgs& l = c->lat;
  const bool sub = kind == VCSGC_SCHED_SUBLATTICE;
  const int q[3] = {sched[0], sched[1], sched[2]};
  if (sub) {
    l.rcp_qx = 1.0f / (float)q[0];
    l.rcp_qy = 1.0f / (float)q[1];
  }
  // geometry (domains per colour, pending slots) and block tables
  long long slots = 0;
  for (int r = 0; r < c->R; ++r) {
    LatGeom g = lattice_geom(c->nx, c->ny, c->nz, sub ? q : nullptr, c->sublattice_d, c->dmax, c->h_geom[r].bits_off,
                             (long long)r * c->dmax);
    g.site_off = c->h_geom[r].site_off;
    c->h_geom[r] = g;
    slots = std::max(slots, g.pend_off + g.dmax);
  }
  CK(cudaMemcpyAsync(const_cast<LatGeom*>(l.geom), c->h_geom.data(), sizeof(LatGeom) * c->R, cudaMemcpyHostToDevice,
                     c->st));
  TRY(dalloc(c, &l.pend, (size_t)slots));
  CK(cudaMemsetAsync(l.pend, 0xFF, sizeof(int) * slots, c->st));
  const int bsz[3] = {64, 128, 256};
  for (int b = 0; b < 3; ++b) {
    std::vector<int2> tab;
    for (int r = 0; r < c->R; ++r) {
      const int nb = std::max(1, (c->h_geom[r].dmax + bsz[b] - 1) / bsz[b]);
      for (int k = 0; k < nb; ++k) tab.push_back(make_int2(r, k * bsz[b]));
    }
    TRY(dalloc(c, &c->blk_tab[b], tab.size()));
    CK(cudaMemcpyAsync(c->blk_tab[b], tab.data(), sizeof(int2) * tab.size(), cudaMemcpyHostToDevice, c->st));
    c->n_blk_tab[b] = (int)tab.size();
  }
  l.dmax = c->dmax;
  select_blk(c);
  fill_args(c);
  // the colour table of the chain's next steps under the new colour count
  TRY(sync_base(c));
  launch_colour_table(l, c->st);
  CK(cudaGetLastError());
  // cluster tilings exist for the sublattice schedule only
  for (int k = 0; k < 5; ++k) {
    c->cl_tiles[k] = nullptr;
    c->cl_smem[k] = 0;
    c->cl_lcap[k] = 0;
  }
  TRY(cluster_setup(c));
  if (c->form == 1 && !cluster_form_usable(c)) c->form = 0;
  CK(cudaStreamSynchronize(c->st));
  return check_device_error(c);
}

int vcsgc_set_schedule(void* ctx, int32_t kind, const int32_t* sched) {
  VCSGC_TRACE("vcsgc_set_schedule");
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || !sched) return VCSGC_ERR_INVALID_ARG;
  return reschedule(c, kind, sched);
}

// In-memory snapshot of a rigid single-lattice chain: species, running
// states, step base.  Restoring it makes the chain continue as if the steps
// since the snapshot had not been taken (the schedule is not part of it).
struct Snap {
  std::vector<uint8_t> types;
  std::vector<RepState> rs;
  long long h_base = 0;
};

static int snap_take(Ctx* c, Snap& s) {
  TRY(sync_bytes(c, -1));
  TRY(refresh_energies(c));
  s.types.resize((size_t)c->R * c->N);
  s.rs.resize(c->R);
  for (int r = 0; r < c->R; ++r)
    CK(cudaMemcpyAsync(s.types.data() + (size_t)r * c->N, c->rep_types[r], c->N, cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(s.rs.data(), c->rs, sizeof(RepState) * c->R, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  s.h_base = c->h_base;
  return check_device_error(c);
}

static int snap_restore(Ctx* c, const Snap& s) {
  TRY(flush(c));
  c->h_base = s.h_base;
  c->base_lag = 0;
  if (c->fast) {
    LatCtl ctl{s.h_base};
    CK(cudaMemcpyAsync(c->lat.ctl, &ctl, sizeof(LatCtl), cudaMemcpyHostToDevice, c->st));
    // no accumulated dn or accepts of any step: the next step starts afresh
    CK(cudaMemsetAsync(c->lat.acc, 0, sizeof(StepAcc) * c->R * 3, c->st));
    launch_colour_table(c->lat, c->st);
    CK(cudaGetLastError());
  } else {
    CK(cudaMemsetAsync(c->acc, 0, sizeof(StepAcc) * c->R, c->st));
  }
  for (int r = 0; r < c->R; ++r) TRY(vcsgc_set_types(c, r, s.types.data() + (size_t)r * c->N));
  CK(cudaMemcpyAsync(c->rs, s.rs.data(), sizeof(RepState) * c->R, cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  c->energy_stale = false;
  drop_graph(c);
  return check_device_error(c);
}

int vcsgc_autotune_schedule(void* ctx, int32_t n_cand, const int32_t* kinds, const int32_t* scheds, int64_t sweeps,
                            double* scores, int32_t* best) {
  VCSGC_TRACE("vcsgc_autotune_schedule");
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || n_cand < 1 || !kinds || !scheds || sweeps < 1 || !scores || !best) return VCSGC_ERR_INVALID_ARG;
  if (c->kind != 0 || !c->subs.empty() || c->multi || c->no_fast)
    return fail(c, VCSGC_ERR_STATE, "schedule autotune: rigid single-lattice contexts only");
  // every candidate starts from the same state; the chain resumes from it
  Snap s0;
  TRY(snap_take(c, s0));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int bi = -1;
  std::vector<vcsgc_observables> o0(c->R), o1(c->R);
  for (int k = 0; k < n_cand; ++k) {
    scores[k] = -1.0;
    if (reschedule(c, kinds[k], scheds + 6 * k) != VCSGC_OK) continue;  // a schedule these lattices refuse
    TRY(snap_restore(c, s0));
    TRY(run_steps(c, sweeps * c->steps_per_sweep));                        // settle under the candidate
    TRY(vcsgc_observables_all(c, o0.data()));
    CK(cudaEventRecord(e0, c->st));
    TRY(run_steps(c, sweeps * c->steps_per_sweep));
    CK(cudaEventRecord(e1, c->st));
    CK(cudaEventSynchronize(e1));
    TRY(vcsgc_observables_all(c, o1.data()));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    long long flips = 0;
    for (int r = 0; r < c->R; ++r) flips += o1[r].flips - o0[r].flips;
    scores[k] = (double)flips / (ms * 1e-3);
    if (bi < 0 || scores[k] > scores[bi]) bi = k;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->err.clear();
  if (bi < 0) return fail(c, VCSGC_ERR_SCHEDULE, "schedule autotune: no candidate schedule applies");
  TRY(reschedule(c, kinds[bi], scheds + 6 * bi));
  TRY(snap_restore(c, s0));
  *best = bi;
  return VCSGC_OK;
}

int vcsgc_set_launch(void* ctx, int32_t form, int32_t block, int32_t variant) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return VCSGC_ERR_INVALID_ARG;
  const bool f0 = form == 0 && (block == 64 || block == 128 || block == 256) && (variant == 0 || variant == 1);
  const bool f1 = form == 1 && (block == 256 || block == 512) && cl_index(variant) >= 0;
  if (!f0 && !f1)
    return fail(c, VCSGC_ERR_INVALID_ARG,
                "launch shape: form 0 with block 64, 128 or 256 and prefetch 0 or 1, or form 1 with block 256 or "
                "512 and 1, 2, 4, 8 or 16 CTAs per cluster");
  if (!c->fast) return fail(c, VCSGC_ERR_STATE, "launch shape: the context is not in the fused form");
  if (f1) {
    const int q = cl_index(variant);
    if (!c->cl_tiles[q] || c->cl_lcap[q] > block * CL_TRIALS_PER_THREAD ||
        (block == 256 && cluster_capacity(variant, 256, c->cl_smem[q]) < 1))
      return fail(c, VCSGC_ERR_STATE, "launch shape: no cluster-resident form of this size for these lattices");
    if (c->lat.da) return fail(c, VCSGC_ERR_STATE, "launch shape: the cluster-resident form has no delayed acceptance");
    c->form = 1;
    c->cl_size = variant;
    c->cl_block = block;
    return VCSGC_OK;
  }
  c->form = 0;
  c->lat.block = block;
  c->lat.prefetch = variant;
  select_blk(c);
  drop_graph(c);
  return VCSGC_OK;
}

int vcsgc_get_launch(void* ctx, int32_t* form, int32_t* block, int32_t* variant) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return VCSGC_ERR_INVALID_ARG;
  const bool f1 = c->fast && cluster_form_usable(c);
  if (form) *form = f1 ? 1 : 0;
  if (block) *block = f1 ? c->cl_block : (c->fast ? c->lat.block : MC_BLOCK);
  if (variant) *variant = f1 ? c->cl_size : (c->fast ? c->lat.prefetch : 0);
  return VCSGC_OK;
}

int vcsgc_cluster_sizes(void* ctx, int32_t* mask) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || !mask) return VCSGC_ERR_INVALID_ARG;
  int m = 0;
  for (int q = 0; q < 5; ++q)
    if (c->cl_tiles[q]) m |= 1 << q;
  *mask = m;
  return VCSGC_OK;
}

const char* vcsgc_last_error(void* ctx) {
  if (!ctx) return g_init_error.c_str();
  return static_cast<Ctx*>(ctx)->err.c_str();
}

int vcsgc_steps(void* ctx, int64_t n) {
  VCSGC_TRACE("vcsgc_steps");
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || n < 0) return VCSGC_ERR_INVALID_ARG;
  return run_steps(c, n);
}

int vcsgc_steps_per_sweep(void* ctx, int64_t* out) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || !out) return VCSGC_ERR_INVALID_ARG;
  *out = c->steps_per_sweep;
  return VCSGC_OK;
}

int vcsgc_sweep(void* ctx, int64_t n) {
  VCSGC_TRACE("vcsgc_sweep");
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || n < 0) return VCSGC_ERR_INVALID_ARG;
  return run_steps(c, n * c->steps_per_sweep);
}

int md_steps(void* ctx, int64_t n) {
  VCSGC_TRACE("md_steps");
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || n < 0) return VCSGC_ERR_INVALID_ARG;
  if (!c->subs.empty()) return fail(c, VCSGC_ERR_STATE, "no MD on a batch");
  TRY(md_run(c, n));
  return check_device_error(c);
}

// Rebuild the SPATIAL schedule from the current positions on the device
// (the same tables as build_schedule: domains by colour, then box index;
// atoms ascending within a domain).  The colour and domain counts do not
// depend on the positions, only the domains' members do.
static int spatial_schedule_device(Ctx* c) {
  const int nb[3] = {c->sched[0], c->sched[1], c->sched[2]}, pp[3] = {c->sched[3], c->sched[4], c->sched[5]};
  const int nblk = nb[0] * nb[1] * nb[2];
  if (!c->sp_dom_of_block) {
    std::vector<int> rank_of(nblk);
    int d = 0;
    const int ncol = pp[0] * pp[1] * pp[2];
    for (int col = 0; col < ncol; ++col)
      for (int b = 0; b < nblk; ++b) {
        const int ibx = b % nb[0], iby = (b / nb[0]) % nb[1], ibz = b / (nb[0] * nb[1]);
        if (((ibz % pp[2]) * pp[1] + (iby % pp[1])) * pp[0] + (ibx % pp[0]) == col) rank_of[b] = d++;
      }
    if (d != c->n_domains) return fail(c, VCSGC_ERR_STATE, "spatial schedule: domain count changed");
    TRY(dalloc(c, &c->sp_dom_of_block, nblk));
    TRY(dalloc(c, &c->sp_dom_of, c->N));
    TRY(dalloc(c, &c->sp_count, d));
    TRY(dalloc(c, &c->sp_cursor, d));
    CK(cudaMemcpyAsync(c->sp_dom_of_block, rank_of.data(), sizeof(int) * nblk, cudaMemcpyHostToDevice, c->st));
    c->sp_ndom = d;
  }
  if (c->dom_sites_cap < c->N) return fail(c, VCSGC_ERR_STATE, "spatial schedule: site table too small");
  launch_spatial_schedule(c->N, c->x, c->y, c->z, c->box, nb, c->sp_dom_of_block, c->sp_ndom, c->sp_dom_of,
                          c->sp_count, c->sp_cursor, c->dom_start, c->dom_sites, c->st);
  CK(cudaGetLastError());
  return VCSGC_OK;
}

int vcsgc_hybrid(void* ctx, int64_t n_cycles, int64_t n_md, int64_t n_mc) {
  VCSGC_TRACE("vcsgc_hybrid");
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || n_cycles < 0 || n_md < 0 || n_mc < 0) return VCSGC_ERR_INVALID_ARG;
  for (int64_t q = 0; q < n_cycles; ++q) {
    TRY(md_run(c, n_md));
    if (c->sched_kind == VCSGC_SCHED_SPATIAL) TRY(spatial_schedule_device(c));
    // positions moved: the tracked energy restarts from a full evaluation
    double e;
    TRY(energy_of(c, 0, &e));
    CK(cudaMemcpyAsync(&c->rs[0].energy, &e, sizeof(double), cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
    TRY(run_steps(c, n_mc));
    c->forces_valid = false;
    TRY(md_forces(c));
  }
  return check_device_error(c);
}

static void fill_observables(const Ctx* c, int r, const RepState& s, vcsgc_observables* o) {
  const RepParams& p = c->h_rp[r];
  std::memset(o, 0, sizeof(*o));
  const double Nr = (double)c->rep_n[r];
  o->n_sites = c->rep_n[r];
  o->n_b = s.n;
  o->c = (double)s.n / Nr;
  o->energy = s.energy;
  o->energy_per_atom = s.energy / Nr;
  o->steps = s.steps;
  o->trials = s.trials;
  o->local_accepts = s.local_acc;
  o->global_trials = s.global_trials;
  o->global_accepts = s.global_acc;
  o->flips = s.flips;
  o->near_ties = s.near_ties;
  o->acc_local = s.trials ? (double)s.local_acc / (double)s.trials : 0.0;
  o->acc_global = s.global_trials ? (double)s.global_acc / (double)s.global_trials : 0.0;
  o->mean_c = s.steps ? s.sum_c / (double)s.steps : o->c;
  o->var_c = s.steps ? std::max(0.0, s.sum_c2 / (double)s.steps - o->mean_c * o->mean_c) : 0.0;
  o->dmu_est = p.phi + 2.0 * p.kappa_p * Nr * o->mean_c;
  o->sweeps = (double)s.trials / Nr;
  o->kappa_p = p.kappa_p;
  o->dmu0 = p.dmu0;
  o->stage1_accepts = s.s1_acc;
}

int observables(void* ctx, int32_t r, vcsgc_observables* o) {
  VCSGC_TRACE("observables");
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || !o || r < 0 || r >= c->R) return VCSGC_ERR_INVALID_ARG;
  TRY(sync_from_multi(c));
  TRY(flush(c));
  TRY(check_device_error(c));
  TRY(refresh_energies(c));
  RepState s;
  CK(cudaMemcpyAsync(&s, c->rs + r, sizeof(RepState), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  fill_observables(c, r, s, o);
  return VCSGC_OK;
}

int vcsgc_observables_all(void* ctx, vcsgc_observables* o) {
  VCSGC_TRACE("vcsgc_observables_all");
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || !o) return VCSGC_ERR_INVALID_ARG;
  TRY(sync_from_multi(c));
  TRY(flush(c));
  TRY(refresh_energies(c));
  // the states and the error word through one pinned buffer, one synchronisation
  const size_t bytes = sizeof(RepState) * c->R + sizeof(unsigned);
  if (c->h_pin_bytes < bytes) {
    if (c->h_pin) cudaFreeHost(c->h_pin);
    c->h_pin = nullptr;
    c->h_pin_bytes = 0;
    CK(cudaMallocHost(&c->h_pin, bytes));
    c->h_pin_bytes = bytes;
  }
  RepState* s = static_cast<RepState*>(c->h_pin);
  unsigned* e = reinterpret_cast<unsigned*>(s + c->R);
  CK(cudaMemcpyAsync(s, c->rs, sizeof(RepState) * c->R, cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(e, c->derr, sizeof(unsigned), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  TRY(device_error_status(c, *e));
  for (int r = 0; r < c->R; ++r) fill_observables(c, r, s[r], o + r);
  return VCSGC_OK;
}

int vcsgc_get_types(void* ctx, int32_t r, uint8_t* out) {
  VCSGC_TRACE("vcsgc_get_types");
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || !out || r < 0 || r >= c->R) return VCSGC_ERR_INVALID_ARG;
  TRY(sync_bytes(c, r));
  CK(cudaMemcpyAsync(out, c->rep_types[r], c->rep_n[r], cudaMemcpyDeviceToHost, c->st));
  return check_device_error(c);
}

// every byte 0 or 1: an OR over 32-byte chunks, tested once at the end
static bool species_ok(const uint8_t* in, long long n) {
  uint64_t acc = 0;
  long long i = 0;
  for (; i + 32 <= n; i += 32) {
    uint64_t w[4];
    std::memcpy(w, in + i, 32);
    acc |= (w[0] | w[1]) | (w[2] | w[3]);
  }
  for (; i + 8 <= n; i += 8) {
    uint64_t w;
    std::memcpy(&w, in + i, 8);
    acc |= w;
  }
  uint8_t tail = 0;
  for (; i < n; ++i) tail |= in[i];
  return !(acc & 0xFEFEFEFEFEFEFEFEull) && !(tail & 0xFEu);
}

// after a device species check: on a bad byte the bits (and so the state)
// were left unchanged; the species bytes are restored from them
static int checked_species(Ctx* c) {
  const int rc = check_device_error(c);
  if (rc == VCSGC_ERR_INVALID_ARG) {
    const std::string msg = c->err;
    TRY(sync_bytes(c, -1));
    TRY(check_device_error(c));
    c->err = msg;
  }
  return rc;
}

int vcsgc_set_types(void* ctx, int32_t r, const uint8_t* in) {
  VCSGC_TRACE("vcsgc_set_types");
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || !in || r < 0 || r >= c->R) return VCSGC_ERR_INVALID_ARG;
  const long long Nr = c->rep_n[r];
  if (c->fast && c->etab) {
    // perfect lattice with one density function: rho does not change; the
    // species are checked, packed, counted and summed on the device
    TRY(flush(c));
    const LatGeom& g = c->h_geom[r];
    CK(cudaMemcpyAsync(c->rep_types[r], in, Nr, cudaMemcpyHostToDevice, c->st));
    launch_species_check(c->rep_types[r], Nr, c->derr, c->st);
    launch_lattice_pack(c->lat, c->d_tptr, r, 1, (long long)g.ny * g.nz * g.W, c->st);
    launch_lattice_energy(c->lat, r, 1, (long long)g.ny * g.nz * g.W, c->etab, c->epart, c->epstride,
                          (int)(c->h_base & 1), c->st);
    CK(cudaGetLastError());
    c->forces_valid = false;
    return checked_species(c);
  }
  if (!species_ok(in, Nr)) return fail(c, VCSGC_ERR_INVALID_ARG, "species must be 0 or 1");
  TRY(sync_from_multi(c));
  TRY(flush(c));
  CK(cudaMemcpyAsync(c->rep_types[r], in, Nr, cudaMemcpyHostToDevice, c->st));
  if (c->fast) {
    long long nb = 0;
    for (long long i = 0; i < Nr; ++i) nb += in[i];
    launch_lattice_pack(c->lat, c->d_tptr, r, 1, (long long)c->h_geom[r].ny * c->h_geom[r].nz * c->h_geom[r].W,
                        c->st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(c->lat.n_start + 2 * r + (c->h_base & 1), &nb, sizeof(long long),
                       cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
  }
  if (!c->subs.empty()) {
    // batch: n and the energy of replica r come from its set-up context
    long long nb = 0;
    for (long long i = 0; i < Nr; ++i) nb += in[i];
    double e = 0.0;
    TRY(energy_of(c, r, &e));
    RepState st;
    CK(cudaMemcpyAsync(&st, c->rs + r, sizeof(RepState), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    st.n = nb;
    st.energy = e;
    CK(cudaMemcpyAsync(c->rs + r, &st, sizeof(RepState), cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
    return check_device_error(c);
  }
  TRY(sync_state_from_types(c, r, in));
  TRY(push_to_multi(c, r, in, nullptr));
  c->forces_valid = false;
  return check_device_error(c);
}

int vcsgc_get_types_all(void* ctx, uint8_t* out) {
  VCSGC_TRACE("vcsgc_get_types_all");
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || !out) return VCSGC_ERR_INVALID_ARG;
  TRY(sync_bytes(c, -1));
  long long off = 0;
  bool contiguous = true;
  for (int r = 0; r < c->R; ++r) {
    if (c->rep_types[r] != c->rep_types[0] + off) contiguous = false;
    off += c->rep_n[r];
  }
  if (contiguous) {
    CK(cudaMemcpyAsync(out, c->rep_types[0], off, cudaMemcpyDeviceToHost, c->st));
  } else {
    off = 0;
    for (int r = 0; r < c->R; ++r) {
      CK(cudaMemcpyAsync(out + off, c->rep_types[r], c->rep_n[r], cudaMemcpyDeviceToHost, c->st));
      off += c->rep_n[r];
    }
  }
  return check_device_error(c);
}

int vcsgc_set_types_all(void* ctx, const uint8_t* in) {
  VCSGC_TRACE("vcsgc_set_types_all");
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || !in) return VCSGC_ERR_INVALID_ARG;
  if (!(c->fast && c->etab)) {
    long long total = 0;
    for (int r = 0; r < c->R; ++r) total += c->rep_n[r];
    if (!species_ok(in, total)) return fail(c, VCSGC_ERR_INVALID_ARG, "species must be 0 or 1");
    long long off = 0;
    for (int r = 0; r < c->R; ++r) {
      TRY(vcsgc_set_types(ctx, r, in + off));
      off += c->rep_n[r];
    }
    return VCSGC_OK;
  }
  TRY(flush(c));
  // one transfer and one check when the replicas' arrays are back to back
  bool contiguous = true;
  long long off = 0;
  for (int r = 0; r < c->R; ++r) {
    if (c->rep_types[r] != c->rep_types[0] + off) contiguous = false;
    off += c->rep_n[r];
  }
  if (contiguous) {
    CK(cudaMemcpyAsync(c->rep_types[0], in, off, cudaMemcpyHostToDevice, c->st));
    launch_species_check(c->rep_types[0], off, c->derr, c->st);
  } else {
    off = 0;
    for (int r = 0; r < c->R; ++r) {
      CK(cudaMemcpyAsync(c->rep_types[r], in + off, c->rep_n[r], cudaMemcpyHostToDevice, c->st));
      launch_species_check(c->rep_types[r], c->rep_n[r], c->derr, c->st);
      off += c->rep_n[r];
    }
  }
  launch_lattice_pack(c->lat, c->d_tptr, 0, c->R, c->max_words, c->st);
  launch_lattice_energy(c->lat, 0, c->R, c->max_words, c->etab, c->epart, c->epstride, (int)(c->h_base & 1),
                        c->st);
  CK(cudaGetLastError());
  c->forces_valid = false;
  return checked_species(c);
}

int vcsgc_get_rho(void* ctx, int32_t r, double* out) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || !out || r < 0 || r >= c->R) return VCSGC_ERR_INVALID_ARG;
  TRY(sync_from_multi(c));
  if (!c->subs.empty()) return vcsgc_get_rho(c->subs[r], 0, out);
  const double* src = c->rho + (c->reembed ? (long long)r * c->N : 0);
  CK(cudaMemcpyAsync(out, src, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->st));
  return check_device_error(c);
}

int vcsgc_delta_e(void* ctx, int32_t r, const int64_t* sites, int64_t n, double* out) {
  VCSGC_TRACE("vcsgc_delta_e");
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || (n > 0 && (!sites || !out)) || n < 0 || r < 0 || r >= c->R) return VCSGC_ERR_INVALID_ARG;
  if (n == 0) return VCSGC_OK;
  TRY(sync_from_multi(c));
  std::vector<int> s32(n);
  for (int64_t q = 0; q < n; ++q) {
    if (sites[q] < 0 || sites[q] >= c->rep_n[r]) return fail(c, VCSGC_ERR_INVALID_ARG, "site index out of range");
    s32[q] = (int)sites[q];
  }
  if (n > c->sites_cap) {
    TRY(dalloc(c, &c->sites_buf, n));
    TRY(dalloc(c, &c->de_buf, n));
    c->sites_cap = (int)n;
  }
  CK(cudaMemcpyAsync(c->sites_buf, s32.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->st));
  if (c->fast) {
    TRY(flush(c));
    launch_lattice_delta_e(c->lat, r, c->sites_buf, (int)n, c->de_buf, c->st);
  } else {
    launch_delta_e_list(c->mc, c->shell, c->reembed, r, c->sites_buf, (int)n, c->de_buf, c->st);
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(out, c->de_buf, sizeof(double) * n, cudaMemcpyDeviceToHost, c->st));
  return check_device_error(c);
}

int vcsgc_energy(void* ctx, int32_t r, double* out) {
  VCSGC_TRACE("vcsgc_energy");
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || !out || r < 0 || r >= c->R) return VCSGC_ERR_INVALID_ARG;
  TRY(sync_from_multi(c));
  return energy_of(c, r, out);
}

int vcsgc_forces(void* ctx, double* fx, double* fy, double* fz) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || !fx || !fy || !fz) return VCSGC_ERR_INVALID_ARG;
  if (!c->subs.empty()) return fail(c, VCSGC_ERR_STATE, "forces are not defined for a batch");
  if (!c->forces_valid) TRY(md_forces(c));
  CK(cudaMemcpyAsync(fx, c->fx, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(fy, c->fy, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(fz, c->fz, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->st));
  return check_device_error(c);
}

int vcsgc_get_md(void* ctx, double* x, double* y, double* z, double* vx, double* vy, double* vz) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return VCSGC_ERR_INVALID_ARG;
  if (!c->subs.empty()) return fail(c, VCSGC_ERR_STATE, "positions are per replica in a batch");
  double* dst[6] = {x, y, z, vx, vy, vz};
  double* src[6] = {c->x, c->y, c->z, c->vx, c->vy, c->vz};
  for (int q = 0; q < 6; ++q) {
    if (!dst[q]) continue;
    if (!src[q]) return fail(c, VCSGC_ERR_STATE, "velocities not set");
    CK(cudaMemcpyAsync(dst[q], src[q], sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->st));
  }
  return check_device_error(c);
}

int vcsgc_set_velocities(void* ctx, const double* vx, const double* vy, const double* vz) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || !vx || !vy || !vz) return VCSGC_ERR_INVALID_ARG;
  if (!c->subs.empty()) return fail(c, VCSGC_ERR_STATE, "no MD on a batch");
  if (c->R != 1) return fail(c, VCSGC_ERR_STATE, "velocities need one replica");
  if (!c->vx) {
    TRY(dalloc(c, &c->vx, c->N));
    TRY(dalloc(c, &c->vy, c->N));
    TRY(dalloc(c, &c->vz, c->N));
  }
  CK(cudaMemcpyAsync(c->vx, vx, sizeof(double) * c->N, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->vy, vy, sizeof(double) * c->N, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->vz, vz, sizeof(double) * c->N, cudaMemcpyHostToDevice, c->st));
  c->have_v = true;
  fill_args(c);
  drop_graph(c);
  return check_device_error(c);
}

int vcsgc_kinetic_energy(void* ctx, double* out) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || !out) return VCSGC_ERR_INVALID_ARG;
  if (!c->have_v) return fail(c, VCSGC_ERR_STATE, "velocities not set");
  launch_kinetic(c->md, c->part, c->st);
  CK(cudaGetLastError());
  const int nb = kinetic_blocks(c->N);
  std::vector<double> h(nb);
  CK(cudaMemcpyAsync(h.data(), c->part, sizeof(double) * nb, cudaMemcpyDeviceToHost, c->st));
  TRY(check_device_error(c));
  double s = 0.0;
  for (double v : h) s += v;
  *out = s;
  return VCSGC_OK;
}

int vcsgc_set_ensemble(void* ctx, int32_t kind, double t_damp, double p_damp, double p_ext_bar, int32_t chain) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || kind < 0 || kind > 2 || chain < 1 || chain > 4) return VCSGC_ERR_INVALID_ARG;
  if (kind && !(t_damp > 0.0)) return fail(c, VCSGC_ERR_INVALID_ARG, "t_damp must be > 0");
  if (kind == 2 && !(p_damp > 0.0)) return fail(c, VCSGC_ERR_INVALID_ARG, "p_damp must be > 0");
  if (kind && (c->kind != 1 || c->R != 1)) return fail(c, VCSGC_ERR_STATE, "needs explicit positions and one replica");
  if (kind == 2 && c->mixed) return fail(c, VCSGC_ERR_STATE, "the barostat needs the FP64 virial (precision FP64)");
  Ctx::Nh& nh = c->nh;
  nh = Ctx::Nh{};
  nh.kind = kind;
  nh.chain = chain;
  nh.t_damp = t_damp;
  nh.p_damp = p_damp;
  nh.p_ext = p_ext_bar * BAR_EV_A3;
  const double kT = KB_EV * c->T_md, nf = 3.0 * (double)c->N;
  for (int k = 0; k < 4; ++k) {
    nh.Q[k] = (k == 0 ? nf : 1.0) * kT * t_damp * t_damp;
    nh.Qb[k] = kT * p_damp * p_damp;
  }
  nh.W = (nf + 3.0) * kT * p_damp * p_damp;
  return VCSGC_OK;
}

int vcsgc_md_state(void* ctx, double* out) {
  VCSGC_TRACE("vcsgc_md_state");
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || !out) return VCSGC_ERR_INVALID_ARG;
  if (c->kind != 1 || c->R != 1 || !c->d_vir) return fail(c, VCSGC_ERR_STATE, "needs explicit positions and one replica");
  double K2 = 0.0, pe = 0.0, vir = 0.0;
  if (c->have_v) TRY(twice_ke_dev(c, &K2));
  TRY(energy_of(c, 0, &pe));
  TRY(md_forces(c));
  TRY(read_virial(c, &vir));
  TRY(check_device_error(c));
  const Ctx::Nh& nh = c->nh;
  const double nf = 3.0 * (double)c->N, kT = KB_EV * c->T_md;
  const double V = c->box[0] * c->box[1] * c->box[2];
  double H = 0.5 * K2 + pe;
  if (nh.kind) {
    for (int k = 0; k < nh.chain; ++k) H += 0.5 * nh.Q[k] * nh.xi[k] * nh.xi[k] + (k == 0 ? nf : 1.0) * kT * nh.eta[k];
    if (nh.kind == 2) {
      H += nh.p_ext * V + 0.5 * nh.W * nh.veps * nh.veps;
      for (int k = 0; k < nh.chain; ++k) H += 0.5 * nh.Qb[k] * nh.xib[k] * nh.xib[k] + kT * nh.etab[k];
    }
  }
  out[0] = 0.5 * K2;
  out[1] = pe;
  out[2] = K2 / (nf * KB_EV);
  out[3] = (K2 + vir) / (3.0 * V) / BAR_EV_A3;
  out[4] = V;
  out[5] = H;
  out[6] = c->box[0];
  out[7] = c->box[1];
  out[8] = c->box[2];
  return VCSGC_OK;
}

int vcsgc_minimize(void* ctx, double ftol, int64_t max_iter, int64_t* iters, double* fmax_out) {
  VCSGC_TRACE("vcsgc_minimize");
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || !(ftol > 0.0) || max_iter < 0) return VCSGC_ERR_INVALID_ARG;
  if (c->kind != 1 || c->R != 1) return fail(c, VCSGC_ERR_STATE, "needs explicit positions and one replica");
  const long long N = c->N, n3 = 3 * N;
  if (!c->cg_x0) {
    TRY(dalloc(c, &c->cg_x0, n3));
    TRY(dalloc(c, &c->cg_d, n3));
    TRY(dalloc(c, &c->cg_f, n3));
    TRY(dalloc(c, &c->cg_g, n3));
  }
  if (!c->cg_part) TRY(dalloc(c, &c->cg_part, std::max(kinetic_blocks(N), dot_blocks(n3))));
  const int nb = dot_blocks(n3);
  std::vector<double> hp(nb);
  auto dot = [&](const double* a, const double* b, double* out) -> int {
    launch_dot(a, b, n3, c->cg_part, c->st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(hp.data(), c->cg_part, sizeof(double) * nb, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    *out = sum_parts(hp);
    return VCSGC_OK;
  };
  auto maxnorm = [&](const double* a, double* out) -> int {
    CK(cudaMemsetAsync(c->max_disp2, 0, sizeof(unsigned long long), c->st));
    launch_max_norm2(a, N, c->max_disp2, c->st);
    unsigned long long bits = 0;
    CK(cudaMemcpyAsync(&bits, c->max_disp2, sizeof(bits), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    double v;
    std::memcpy(&v, &bits, sizeof(v));
    *out = std::sqrt(v);
    return VCSGC_OK;
  };
  auto copy_pos = [&](double* dst) -> int {
    CK(cudaMemcpyAsync(dst, c->x, sizeof(double) * N, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpyAsync(dst + N, c->y, sizeof(double) * N, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpyAsync(dst + 2 * N, c->z, sizeof(double) * N, cudaMemcpyDeviceToDevice, c->st));
    return VCSGC_OK;
  };
  // forces at x0 + alpha d into g (neighbour list rebuilt past half the skin)
  auto eval_at = [&](double alpha, double* g) -> int {
    CK(cudaMemsetAsync(c->max_disp2, 0, sizeof(unsigned long long), c->st));
    launch_cg_place(c->md, c->cg_x0, c->cg_d, alpha, c->st);
    CK(cudaGetLastError());
    unsigned long long bits = 0;
    CK(cudaMemcpyAsync(&bits, c->max_disp2, sizeof(bits), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    double d2;
    std::memcpy(&d2, &bits, sizeof(d2));
    if (d2 > 0.25 * c->skin * c->skin) TRY(md_rebuild(c));
    TRY(md_forces(c));
    CK(cudaMemcpyAsync(g, c->fx, sizeof(double) * N, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpyAsync(g + N, c->fy, sizeof(double) * N, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpyAsync(g + 2 * N, c->fz, sizeof(double) * N, cudaMemcpyDeviceToDevice, c->st));
    return VCSGC_OK;
  };
  // Polak-Ribiere conjugate gradients; the line search finds a zero of
  // phi'(alpha) = -F(x0 + alpha d) . d (extension, then regula falsi)
  TRY(copy_pos(c->cg_x0));
  CK(cudaMemsetAsync(c->cg_d, 0, sizeof(double) * n3, c->st));
  TRY(eval_at(0.0, c->cg_f));
  CK(cudaMemcpyAsync(c->cg_d, c->cg_f, sizeof(double) * n3, cudaMemcpyDeviceToDevice, c->st));
  double ff = 0.0, step = 0.0, fmax = 0.0;
  TRY(dot(c->cg_f, c->cg_f, &ff));
  int64_t it = 0;
  int converged = 0;
  for (; it < max_iter; ++it) {
    TRY(maxnorm(c->cg_f, &fmax));
    if (fmax < ftol) {
      converged = 1;
      break;
    }
    double dmax = 0.0, p0 = 0.0, p1 = 0.0;
    TRY(maxnorm(c->cg_d, &dmax));
    TRY(dot(c->cg_f, c->cg_d, &p0));
    p0 = -p0;
    const double pstart = std::fabs(p0);
    double a0 = 0.0, a1 = step > 0.0 ? step : 0.05 / dmax;
    if (a1 * dmax > 0.2) a1 = 0.2 / dmax;
    TRY(eval_at(a1, c->cg_g));
    TRY(dot(c->cg_g, c->cg_d, &p1));
    p1 = -p1;
    for (int ls = 0; ls < 30 && p1 < 0.0 && std::fabs(p1) > 1e-3 * pstart; ++ls) {
      a0 = a1;
      p0 = p1;
      a1 *= 2.0;
      TRY(eval_at(a1, c->cg_g));
      TRY(dot(c->cg_g, c->cg_d, &p1));
      p1 = -p1;
    }
    for (int ls = 0; ls < 40 && std::fabs(p1) > 1e-3 * pstart && p1 > 0.0; ++ls) {
      const double a2 = a0 - p0 * (a1 - a0) / (p1 - p0);
      double p2 = 0.0;
      TRY(eval_at(a2, c->cg_g));
      TRY(dot(c->cg_g, c->cg_d, &p2));
      p2 = -p2;
      if (p2 < 0.0) {
        a0 = a2;
        p0 = p2;
        if (std::fabs(p2) <= 1e-3 * pstart) {
          a1 = a2;
          p1 = p2;
        }
      } else {
        a1 = a2;
        p1 = p2;
      }
    }
    if (p1 > 0.0 && std::fabs(p1) > 1e-3 * pstart) TRY(eval_at(a1, c->cg_g));
    step = a1;
    TRY(copy_pos(c->cg_x0));
    double gg = 0.0, gf = 0.0, gd = 0.0;
    TRY(dot(c->cg_g, c->cg_g, &gg));
    TRY(dot(c->cg_g, c->cg_f, &gf));
    const double beta = std::max(0.0, (gg - gf) / ff);
    launch_axpby(c->cg_d, c->cg_g, beta, n3, c->st);
    CK(cudaGetLastError());
    TRY(dot(c->cg_g, c->cg_d, &gd));
    if (gd <= 0.0) CK(cudaMemcpyAsync(c->cg_d, c->cg_g, sizeof(double) * n3, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpyAsync(c->cg_f, c->cg_g, sizeof(double) * n3, cudaMemcpyDeviceToDevice, c->st));
    ff = gg;
  }
  // the tracked energy restarts from the relaxed positions
  double e = 0.0;
  TRY(energy_of(c, 0, &e));
  CK(cudaMemcpyAsync(&c->rs[0].energy, &e, sizeof(double), cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (iters) *iters = it;
  if (fmax_out) *fmax_out = fmax;
  (void)converged;
  return check_device_error(c);
}

// ------------------------------------------------------ checkpoint / resume
// File: "VCSGCCK1", a header of int64 (N, R, kind, schedule, fast,
// sizeof(RepState), sizeof(Nh), have_v), rep_n[R], the species of every
// replica, the RepState array, the fused step base, the MD step, the box,
// then (explicit positions) x, y, z, (velocities) vx, vy, vz, and the
// Nose-Hoover state.  Host byte order.
static const char kCkMagic[8] = {'V', 'C', 'S', 'G', 'C', 'C', 'K', '1'};

int vcsgc_save(void* ctx, const char* path) {
  VCSGC_TRACE("vcsgc_save");
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || !path) return VCSGC_ERR_INVALID_ARG;
  TRY(sync_from_multi(c));
  TRY(sync_bytes(c, -1));
  TRY(refresh_energies(c));
  long long tot = 0;
  for (int r = 0; r < c->R; ++r) tot += c->rep_n[r];
  std::vector<uint8_t> types(tot);
  long long off = 0;
  for (int r = 0; r < c->R; ++r) {
    CK(cudaMemcpyAsync(types.data() + off, c->rep_types[r], c->rep_n[r], cudaMemcpyDeviceToHost, c->st));
    off += c->rep_n[r];
  }
  std::vector<RepState> rs(c->R);
  CK(cudaMemcpyAsync(rs.data(), c->rs, sizeof(RepState) * c->R, cudaMemcpyDeviceToHost, c->st));
  std::vector<double> md;
  const bool pos = c->kind == 1;
  if (pos) {
    md.resize((c->have_v ? 6 : 3) * (size_t)c->N);
    double* dst[6] = {c->x, c->y, c->z, c->vx, c->vy, c->vz};
    for (int q = 0; q < (c->have_v ? 6 : 3); ++q)
      CK(cudaMemcpyAsync(md.data() + q * c->N, dst[q], sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->st));
  }
  CK(cudaStreamSynchronize(c->st));
  TRY(check_device_error(c));
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(c, VCSGC_ERR_INVALID_ARG, std::string("cannot open ") + path);
  const long long hdr[8] = {c->N, c->R, c->kind, c->sched_kind, c->fast ? 1 : 0, (long long)sizeof(RepState),
                            (long long)sizeof(Ctx::Nh), c->have_v ? 1 : 0};
  bool ok = std::fwrite(kCkMagic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
            std::fwrite(c->rep_n.data(), sizeof(long long), c->R, f) == (size_t)c->R &&
            std::fwrite(types.data(), 1, tot, f) == (size_t)tot &&
            std::fwrite(rs.data(), sizeof(RepState), c->R, f) == (size_t)c->R &&
            std::fwrite(&c->h_base, sizeof(long long), 1, f) == 1 && std::fwrite(&c->md_step, sizeof(long long), 1, f) == 1 &&
            std::fwrite(c->box, sizeof(double), 3, f) == 3 &&
            (md.empty() || std::fwrite(md.data(), sizeof(double), md.size(), f) == md.size()) &&
            std::fwrite(&c->nh, sizeof(Ctx::Nh), 1, f) == 1;
  ok = (std::fclose(f) == 0) && ok;
  return ok ? VCSGC_OK : fail(c, VCSGC_ERR_INVALID_ARG, std::string("write failed: ") + path);
}

int vcsgc_load(void* ctx, const char* path) {
  VCSGC_TRACE("vcsgc_load");
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || !path) return VCSGC_ERR_INVALID_ARG;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(c, VCSGC_ERR_INVALID_ARG, std::string("cannot open ") + path);
  char magic[8];
  long long hdr[8];
  std::vector<long long> rep_n(c->R);
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kCkMagic, 8) == 0 &&
            std::fread(hdr, sizeof(hdr), 1, f) == 1;
  ok = ok && hdr[0] == c->N && hdr[1] == c->R && hdr[2] == c->kind && hdr[3] == c->sched_kind &&
       hdr[4] == (c->fast ? 1 : 0) && hdr[5] == (long long)sizeof(RepState) && hdr[6] == (long long)sizeof(Ctx::Nh);
  ok = ok && std::fread(rep_n.data(), sizeof(long long), c->R, f) == (size_t)c->R && rep_n == c->rep_n;
  long long tot = 0;
  for (long long v : rep_n) tot += v;
  std::vector<uint8_t> types(ok ? tot : 0);
  std::vector<RepState> rs(c->R);
  long long h_base = 0, md_step = 0;
  double box[3] = {0, 0, 0};
  const bool pos = c->kind == 1, vel = ok && hdr[7] == 1;
  std::vector<double> md(pos ? (vel ? 6 : 3) * (size_t)c->N : 0);
  Ctx::Nh nh;
  ok = ok && std::fread(types.data(), 1, tot, f) == (size_t)tot &&
       std::fread(rs.data(), sizeof(RepState), c->R, f) == (size_t)c->R &&
       std::fread(&h_base, sizeof(long long), 1, f) == 1 && std::fread(&md_step, sizeof(long long), 1, f) == 1 &&
       std::fread(box, sizeof(double), 3, f) == 3 &&
       (md.empty() || std::fread(md.data(), sizeof(double), md.size(), f) == md.size()) &&
       std::fread(&nh, sizeof(Ctx::Nh), 1, f) == 1;
  std::fclose(f);
  for (int q = 0; q < 3 && ok && pos; ++q) ok = std::isfinite(box[q]) && box[q] > 2.0 * c->rc;
  if (!ok) return fail(c, VCSGC_ERR_INVALID_ARG, "checkpoint does not match this context (sizes, schedule or form)");
  TRY(flush(c));
  CK(cudaStreamSynchronize(c->st));
  // step base (fused form) first: the species upload writes n at its parity
  c->h_base = h_base;
  c->base_lag = 0;
  if (c->fast) {
    LatCtl ctl{h_base};
    CK(cudaMemcpyAsync(c->lat.ctl, &ctl, sizeof(LatCtl), cudaMemcpyHostToDevice, c->st));
    launch_colour_table(c->lat, c->st);
    CK(cudaGetLastError());
  }
  if (pos) {
    for (int q = 0; q < 3; ++q) c->box[q] = box[q];
    // positions into [0, L) as at init (the kernels' minimum image needs it)
    for (int q = 0; q < 3; ++q)
      for (long long i = 0; i < c->N; ++i) {
        double& v = md[q * c->N + i];
        v -= c->box[q] * std::floor(v / c->box[q]);
        if (!(v < c->box[q]) || v < 0.0) v = 0.0;
      }
    double* dst[3] = {c->x, c->y, c->z};
    for (int q = 0; q < 3; ++q)
      CK(cudaMemcpyAsync(dst[q], md.data() + q * c->N, sizeof(double) * c->N, cudaMemcpyHostToDevice, c->st));
    fill_args(c);
    TRY(md_rebuild(c));
    if (vel) TRY(vcsgc_set_velocities(c, md.data() + 3 * c->N, md.data() + 4 * c->N, md.data() + 5 * c->N));
    c->md_step = md_step;
    c->nh = nh;
  }
  long long off = 0;
  for (int r = 0; r < c->R; ++r) {
    TRY(vcsgc_set_types(c, r, types.data() + off));
    off += rep_n[r];
  }
  // counters, step and the tracked energy exactly as saved
  CK(cudaMemcpyAsync(c->rs, rs.data(), sizeof(RepState) * c->R, cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  off = 0;
  for (int r = 0; r < c->R; ++r) {
    TRY(push_to_multi(c, r, types.data() + off, &rs[r]));
    off += rep_n[r];
  }
  c->energy_stale = false;
  c->forces_valid = false;
  fill_args(c);
  return check_device_error(c);
}

int vcsgc_profile_steps(void* ctx, int64_t n, double* ms_propose, double* ms_commit) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || n < 1 || !ms_propose || !ms_commit) return VCSGC_ERR_INVALID_ARG;
  if (c->multi || (c->fast && cluster_form_usable(c))) {
    // one persistent launch of n steps: its whole time is reported as propose
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    TRY(flush(c));
    CK(cudaEventRecord(e0, c->st));
    TRY(c->multi ? run_steps(c, n) : run_steps_cluster(c, n));
    CK(cudaEventRecord(e1, c->st));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_propose = ms;
    *ms_commit = 0.0;
    return check_device_error(c);
  }
  if (c->fast) TRY(sync_base(c));
  std::vector<cudaEvent_t> ev(2 * n + 1);
  for (auto& e : ev) CK(cudaEventCreate(&e));
  CK(cudaEventRecord(ev[0], c->st));
  for (int64_t q = 0; q < n; ++q) {
    if (c->fast) {
      launch_lattice_step(c->lat, (int)q, true, c->st);
      CK(cudaEventRecord(ev[2 * q + 1], c->st));
      CK(cudaEventRecord(ev[2 * q + 2], c->st));
    } else {
      launch_colour_step(c->mc, c->shell, c->reembed, c->st, 1);
      CK(cudaEventRecord(ev[2 * q + 1], c->st));
      launch_colour_step(c->mc, c->shell, c->reembed, c->st, 2);
      CK(cudaEventRecord(ev[2 * q + 2], c->st));
    }
  }
  if (c->fast) {
    launch_lattice_advance(c->lat, (int)n, c->st);
    c->h_base += n;
    c->pending = true;
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->st));
  double tp = 0.0, tc = 0.0;
  for (int64_t q = 0; q < n; ++q) {
    float a = 0.f, b = 0.f;
    CK(cudaEventElapsedTime(&a, ev[2 * q], ev[2 * q + 1]));
    CK(cudaEventElapsedTime(&b, ev[2 * q + 1], ev[2 * q + 2]));
    tp += a;
    tc += b;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  *ms_propose = tp;
  *ms_commit = tc;
  return check_device_error(c);
}

int vcsgc_neighbours(void* ctx, int64_t i, int32_t* out, int32_t cap, int32_t* count) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || !out || !count || i < 0 || i >= c->N || cap < 0) return VCSGC_ERR_INVALID_ARG;
  if (!c->subs.empty()) return fail(c, VCSGC_ERR_STATE, "neighbour lists are per replica in a batch");
  int cnt = 0;
  CK(cudaMemcpyAsync(&cnt, c->nbr_cnt + i, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  *count = cnt;
  const int m = std::min(cnt, (int)cap);
  if (m > 0) {
    CK(cudaMemcpyAsync(out, c->nbr + i * c->K, sizeof(int) * m, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
  }
  return VCSGC_OK;
}

// ---- delayed acceptance (the learned first stage)
static bool da_neighbourhood(const Ctx* c) {
  // the descriptor's five BCC shells (8, 6, 12, 24, 8 sites) in 13 rows per basis
  if (!c->fast || c->lat.n_shells != 5 || c->lat.n_rows[0] != 13 || c->lat.n_rows[1] != 13) return false;
  int zs[5] = {0, 0, 0, 0, 0};
  for (int sh : c->offset_shell) zs[sh]++;
  return zs[0] == 8 && zs[1] == 6 && zs[2] == 12 && zs[3] == 24 && zs[4] == 8;
}

int vcsgc_features(void* ctx, float* d_X, float* d_Y) {
  VCSGC_TRACE("vcsgc_features");
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c || !d_X || !d_Y) return VCSGC_ERR_INVALID_ARG;
  if (c->multi) {
    // species-dependent densities: the two-species multicomponent object
    // holds the state (same rows: replica after replica in site order)
    const int rc = vcsgc_multi_features(c->multi, d_X, d_Y);
    return rc == VCSGC_OK ? VCSGC_OK : fail(c, rc, vcsgc_multi_last_error(c->multi));
  }
  if (!da_neighbourhood(c))
    return fail(c, VCSGC_ERR_STATE, "features need the fused rigid-lattice form with the 5-shell BCC neighbourhood");
  TRY(flush(c));
  long long max_sites = 0;
  for (const LatGeom& g : c->h_geom) max_sites = std::max(max_sites, g.n_sites);
  launch_lattice_features(c->lat, max_sites, d_X, d_Y, c->st);
  CK(cudaGetLastError());
  return check_device_error(c);
}

int vcsgc_set_surrogate(void* ctx, void* mlp) {
  Ctx* c = static_cast<Ctx*>(ctx);
  if (!c) return VCSGC_ERR_INVALID_ARG;
  if (c->multi) {
    const int rc = vcsgc_multi_set_surrogate(c->multi, mlp);
    return rc == VCSGC_OK ? VCSGC_OK : fail(c, rc, vcsgc_multi_last_error(c->multi));
  }
  if (!mlp) {
    TRY(flush(c));
    CK(cudaStreamSynchronize(c->st));
    c->lat.da = 0;
    drop_graph(c);
    return VCSGC_OK;
  }
  if (!da_neighbourhood(c))
    return fail(c, VCSGC_ERR_STATE,
                "delayed acceptance needs the fused rigid-lattice form with the 5-shell BCC neighbourhood");
  MlpBuf src{};
  if (!mlp_object_buffers(mlp, &src)) return VCSGC_ERR_INVALID_ARG;
  if (!c->sur.w1f) {
    TRY(dalloc(c, &c->sur.w1f, MLP_W1F));
    TRY(dalloc(c, &c->sur.w2f, MLP_W2F));
    TRY(dalloc(c, &c->sur.w2tf, MLP_W2F));
    TRY(dalloc(c, &c->sur.vec, MLP_VEC));
  }
  // the surrogate's own stream may still be writing its fragments
  CK(cudaStreamSynchronize(mlp_object_stream(mlp)));
  TRY(flush(c));
  CK(cudaMemcpyAsync(c->sur.w1f, src.w1f, sizeof(uint2) * MLP_W1F, cudaMemcpyDeviceToDevice, c->st));
  CK(cudaMemcpyAsync(c->sur.w2f, src.w2f, sizeof(uint2) * MLP_W2F, cudaMemcpyDeviceToDevice, c->st));
  CK(cudaMemcpyAsync(c->sur.w2tf, src.w2tf, sizeof(uint2) * MLP_W2F, cudaMemcpyDeviceToDevice, c->st));
  CK(cudaMemcpyAsync(c->sur.vec, src.vec, sizeof(float) * MLP_VEC, cudaMemcpyDeviceToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  c->lat.mlp = mlp_view(c->sur);
  c->lat.da = 1;
  drop_graph(c);  // the captured steps hold the arguments by value
  return VCSGC_OK;
}

}  // extern "C"
