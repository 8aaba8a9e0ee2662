// C ABI of the multicomponent colour step (declarations and the method's
// statement in include/vcsgc.h).  One context holds R replicas of one rigid
// BCC lattice with K <= 4 species; every colour step is a propose and a
// commit launch, captured as CUDA graphs of 64 steps.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.h"
#include "multi.cuh"
#include "screen.h"
#include "trace.h"
#include "vcsgc.h"

namespace vcsgc {
namespace {

struct Multi {
  int device = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::string err;
  int R = 1, K = 2;
  int nx = 0, ny = 0, nz = 0;
  double a = 0, rc = 0;
  long long N = 0;
  long long steps_per_sweep = 1;
  MultiArgs args{};
  std::vector<void*> allocs;
  std::vector<MRepParams> h_rp;
  double* part = nullptr;
  int n_part = 0;
  long long* d_sites = nullptr;
  uint8_t* d_to = nullptr;
  double* d_out = nullptr;
  long long buf_n = 0;
  cudaGraphExec_t graph = nullptr;
  long long* d_base = nullptr;  // fused form: device step base
  long long h_base = 0;         // its host mirror
  // delayed acceptance: the context's copy of the surrogate's fragments;
  // the per-site shell counts are rebuilt from the species before the next
  // use after any change the commit did not track
  MlpBuf sur{};
  bool nbc_stale = true;
  // screened form: the accumulator of the next step (zero sums, the counts
  // at its start) is rewritten from the replicas' states before the next
  // run after the host changed a state or the step base
  bool acc_stale = true;
  // screened form: F_t at the middle of the reachable densities, the
  // offset of species t's FP32 embedding table
  std::vector<double> fref;
};

#define MCK(call)                                                                      \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      m->err = std::string(#call) + ": " + cudaGetErrorString(e_);                     \
      return VCSGC_ERR_CUDA;                                                           \
    }                                                                                  \
  } while (0)
#define MTRY(expr)                     \
  do {                                 \
    int rc_ = (expr);                  \
    if (rc_ != VCSGC_OK) return rc_;   \
  } while (0)

int mfail(Multi* m, int code, const std::string& msg) {
  m->err = msg;
  return code;
}

template <typename T>
int malloc_dev(Multi* m, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, sizeof(T) * std::max<size_t>(count, 1));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return mfail(m, VCSGC_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  m->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return VCSGC_OK;
}

int device_error(Multi* m) {
  unsigned e = 0;
  MCK(cudaMemcpyAsync(&e, m->args.err, sizeof(unsigned), cudaMemcpyDeviceToHost, m->st));
  MCK(cudaStreamSynchronize(m->st));
  if (!e) return VCSGC_OK;
  MCK(cudaMemsetAsync(m->args.err, 0, sizeof(unsigned), m->st));
  MCK(cudaStreamSynchronize(m->st));
  if (e & ERRF_TABLE) return mfail(m, VCSGC_ERR_TABLE_RANGE, "r or rho outside the EAM table grid");
  return mfail(m, VCSGC_ERR_NONFINITE, "non-finite energy difference");
}

// Spline of n samples on the grid j h, coefficients built on the device
int make_spline(Multi* m, const double* y, const double* dy, int n, double h, Spline& s) {
  double *yd = nullptr, *md = nullptr;
  Cubic* c = nullptr;
  MTRY(malloc_dev(m, &yd, n));
  MCK(cudaMemcpyAsync(yd, y, sizeof(double) * n, cudaMemcpyHostToDevice, m->st));
  if (dy) {
    MTRY(malloc_dev(m, &md, n));
    MCK(cudaMemcpyAsync(md, dy, sizeof(double) * n, cudaMemcpyHostToDevice, m->st));
  }
  MTRY(malloc_dev(m, &c, n - 1));
  launch_spline_coeffs(yd, md, n, h, c, m->st);
  MCK(cudaGetLastError());
  s.c = c;
  s.inv_h = 1.0 / h;
  s.xmax = (n - 1) * h;
  s.n_int = n - 1;
  return VCSGC_OK;
}

// energy of replica r from its species and densities (compensated sum of
// the block partials)
int energy_of(Multi* m, int r, double* out) {
  launch_multi_energy(m->args, r, 1, m->part, m->st);
  MCK(cudaGetLastError());
  std::vector<double> h(m->n_part);
  MCK(cudaMemcpyAsync(h.data(), m->part, sizeof(double) * m->n_part, cudaMemcpyDeviceToHost, m->st));
  MCK(cudaStreamSynchronize(m->st));
  MTRY(device_error(m));
  double s = 0.0, c = 0.0;
  for (double v : h) {
    const double t = s + v;
    c += std::fabs(s) >= std::fabs(v) ? (s - t) + v : (v - t) + s;
    s = t;
  }
  *out = s + c;
  return VCSGC_OK;
}

int flush(Multi* m);

// densities, counts and energy of replica r from host species t
int load_replica(Multi* m, int r, const uint8_t* t, bool reset_counters) {
  for (long long i = 0; i < m->N; ++i)
    if (t[i] >= m->K) return mfail(m, VCSGC_ERR_INVALID_ARG, "species value >= K");
  MTRY(flush(m));
  m->nbc_stale = true;
  m->acc_stale = true;
  MCK(cudaMemcpyAsync(m->args.types + (long long)r * m->N, t, m->N, cudaMemcpyHostToDevice, m->st));
  launch_multi_rho(m->args, r, 1, m->st);
  MCK(cudaGetLastError());
  double e = 0.0;
  MTRY(energy_of(m, r, &e));
  MRepState s{};
  if (!reset_counters) {
    MCK(cudaMemcpyAsync(&s, m->args.rs + r, sizeof(MRepState), cudaMemcpyDeviceToHost, m->st));
    MCK(cudaStreamSynchronize(m->st));
  }
  for (int al = 0; al < MK_MAX; ++al) s.cnt[al] = 0;
  for (long long i = 0; i < m->N; ++i) s.cnt[t[i]]++;
  s.energy = e;
  if (reset_counters) s.fin_step = -1;
  if (m->args.fused)
    MCK(cudaMemcpyAsync(m->args.nstart + (2 * r + (int)(m->h_base & 1)) * MK_MAX, s.cnt, sizeof(long long) * MK_MAX,
                        cudaMemcpyHostToDevice, m->st));
  MCK(cudaMemcpyAsync(m->args.rs + r, &s, sizeof(MRepState), cudaMemcpyHostToDevice, m->st));
  MCK(cudaStreamSynchronize(m->st));
  return VCSGC_OK;
}

// fused form: commit the last proposed step and fold it into the state
int flush(Multi* m) {
  if (!m->args.fused || m->h_base == 0) return VCSGC_OK;
  launch_multi_fused(m->args, 0, false, m->st);
  MCK(cudaGetLastError());
  return VCSGC_OK;
}

int run_steps_fused(Multi* m, long long n) {
  const int G = 64;
  if (n >= G && !m->graph) {
    cudaGraph_t g;
    MCK(cudaStreamBeginCapture(m->st, cudaStreamCaptureModeThreadLocal));
    for (int q = 0; q < G; ++q) launch_multi_fused(m->args, q, true, m->st);
    launch_multi_advance(m->d_base, G, m->st);
    cudaError_t e1 = cudaGetLastError();
    MCK(cudaStreamEndCapture(m->st, &g));
    if (e1 != cudaSuccess) {
      cudaGraphDestroy(g);
      return mfail(m, VCSGC_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e1));
    }
    cudaError_t e2 = cudaGraphInstantiate(&m->graph, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) return mfail(m, VCSGC_ERR_CUDA, std::string("graph: ") + cudaGetErrorString(e2));
  }
  for (; n >= G; n -= G) {
    MCK(cudaGraphLaunch(m->graph, m->st));
    m->h_base += G;
  }
  if (n > 0) {
    for (long long q = 0; q < n; ++q) launch_multi_fused(m->args, (int)q, true, m->st);
    launch_multi_advance(m->d_base, (int)n, m->st);
    m->h_base += n;
  }
  MCK(cudaGetLastError());
  return VCSGC_OK;
}

// delayed acceptance: per-site shell counts from the species, if stale
int nbc_fresh(Multi* m) {
  if (!m->nbc_stale) return VCSGC_OK;
  launch_multi_nbc(m->args, m->st);
  MCK(cudaGetLastError());
  m->nbc_stale = false;
  return VCSGC_OK;
}

// screened form: every replica's accumulator of step h_base from its state
int screen_acc_ready(Multi* m) {
  if (!m->args.screen || !m->acc_stale) return VCSGC_OK;
  std::vector<MRepState> s(m->R);
  MCK(cudaMemcpyAsync(s.data(), m->args.rs, sizeof(MRepState) * m->R, cudaMemcpyDeviceToHost, m->st));
  MCK(cudaStreamSynchronize(m->st));
  std::vector<MStepAcc> acc(m->R);
  for (int r = 0; r < m->R; ++r) {
    acc[r] = MStepAcc{};
    for (int al = 0; al < MK_MAX; ++al) acc[r].cnt[al] = s[r].cnt[al];
  }
  const int par = (int)(m->h_base & 1);
  for (int r = 0; r < m->R; ++r)
    MCK(cudaMemcpyAsync(m->args.acc + 2 * r + par, &acc[r], sizeof(MStepAcc), cudaMemcpyHostToDevice, m->st));
  MCK(cudaMemcpyAsync(m->d_base, &m->h_base, sizeof(long long), cudaMemcpyHostToDevice, m->st));
  MCK(cudaStreamSynchronize(m->st));
  m->acc_stale = false;
  return VCSGC_OK;
}

int run_steps(Multi* m, long long n) {
  if (m->args.fused) return run_steps_fused(m, n);
  MTRY(screen_acc_ready(m));
  if (m->args.da) MTRY(nbc_fresh(m));
  // steps without delayed acceptance do not keep the counts
  else if (n > 0) m->nbc_stale = true;
  const int G = 64;
  if (n >= G && !m->graph) {
    cudaGraph_t g;
    MCK(cudaStreamBeginCapture(m->st, cudaStreamCaptureModeThreadLocal));
    for (int q = 0; q < G; ++q) launch_multi_step(m->args, q, m->st, q > 0);
    if (m->args.screen) launch_multi_advance(m->d_base, G, m->st);
    cudaError_t e1 = cudaGetLastError();
    MCK(cudaStreamEndCapture(m->st, &g));
    if (e1 != cudaSuccess) {
      cudaGraphDestroy(g);
      return mfail(m, VCSGC_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e1));
    }
    cudaError_t e2 = cudaGraphInstantiate(&m->graph, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) return mfail(m, VCSGC_ERR_CUDA, std::string("graph: ") + cudaGetErrorString(e2));
  }
  for (; n >= G; n -= G) {
    MCK(cudaGraphLaunch(m->graph, m->st));
    m->h_base += G;
  }
  if (n > 0) {
    for (long long q = 0; q < n; ++q) launch_multi_step(m->args, (int)q, m->st, q > 0);
    // the base is read before the next propose's wait: it moves by an
    // ordinary launch, and the next run starts with an ordinary launch
    if (m->args.screen) launch_multi_advance(m->d_base, (int)n, m->st);
    m->h_base += n;
  }
  MCK(cudaGetLastError());
  return VCSGC_OK;
}

void drop_graph(Multi* m) {
  if (m->graph) cudaGraphExecDestroy(m->graph);
  m->graph = nullptr;
}

void destroy(Multi* m) {
  if (!m) return;
  if (m->st) cudaStreamSynchronize(m->st);
  if (m->graph) cudaGraphExecDestroy(m->graph);
  for (void* p : m->allocs) cudaFree(p);
  if (m->own_stream && m->st) cudaStreamDestroy(m->st);
  delete m;
}

thread_local std::string g_init_err;

// Tables and error bound of the FP32 screen with re-embedding (the bound:
// screen.h).
int screen_setup(Multi* m, const std::vector<double>& hFd) {
  MultiArgs& a = m->args;
  const int n = a.embed[0].n_int;
  for (int al = 1; al < m->K; ++al)
    if (a.embed[al].n_int != n || a.embed[al].inv_h != a.embed[0].inv_h)
      return mfail(m, VCSGC_ERR_INVALID_ARG, "embedding tables on different grids");
  float4* e32 = nullptr;
  MTRY(malloc_dev(m, &e32, (size_t)m->K * n));
  std::vector<std::vector<Cubic>> hc((size_t)m->K, std::vector<Cubic>((size_t)n));
  for (int al = 0; al < m->K; ++al)
    MCK(cudaMemcpyAsync(hc[al].data(), a.embed[al].c, sizeof(Cubic) * n, cudaMemcpyDeviceToHost, m->st));
  MCK(cudaStreamSynchronize(m->st));
  const double h = 1.0 / a.embed[0].inv_h;
  double dmax = 0.0;
  for (int s = 0; s < a.n_sh; ++s)
    for (int x = 0; x < m->K; ++x)
      for (int y = 0; y < m->K; ++y) dmax = std::max(dmax, std::fabs(hFd[s * m->K + y] - hFd[s * m->K + x]));
  // Every site of the rigid five-shell lattice has the same 58 neighbours,
  // so its density lies between the sums of each shell's smallest and
  // largest f, and a screened argument (a density plus one shell's f_b -
  // f_a) within dmax of that (with a margin for float rounding and the
  // FP64 densities' accumulated updates), clipped to the grid.  Arguments
  // outside go to FP64.
  std::vector<int> n_s((size_t)a.n_sh, 0);
  for (int k = 0; k < a.n_off; ++k) n_s[a.off[k].w]++;
  double rmin = 0.0, rmax = 0.0;
  for (int s = 0; s < a.n_sh; ++s) {
    double fl = hFd[s * m->K], fh = hFd[s * m->K];
    for (int x = 1; x < m->K; ++x) {
      fl = std::min(fl, hFd[s * m->K + x]);
      fh = std::max(fh, hFd[s * m->K + x]);
    }
    rmin += n_s[s] * fl;
    rmax += n_s[s] * fh;
  }
  const double xmax = n * h * (1.0 - 1e-6);
  double lo = std::max(h, (rmin - dmax) * (1.0 - 1e-5));
  double hi = std::min(xmax, (rmax + dmax) * (1.0 + 1e-5));
  if (!(lo < hi)) {
    // the reachable densities lie beyond the grid: the whole grid's range
    // (every trial then takes the FP64 path, which reports the table range)
    lo = std::max(h, n * h / 20.0);
    hi = xmax;
  }
  // FP32 tables of F_t - F_t(rho_mid): differences of one species' values
  // are unchanged, the own-site change gets F_b(rho_mid) - F_a(rho_mid)
  // back through the screen's constant, and the coefficients' rounding
  // (the bound's largest term) scales with the smaller values
  const double rmid = std::min(hi, std::max(lo, 0.5 * (rmin + rmax)));
  std::vector<std::vector<Cubic>> hs = hc;
  std::vector<float4> h32((size_t)m->K * n);
  m->fref.assign((size_t)m->K, 0.0);
  for (int al = 0; al < m->K; ++al) {
    const int jm = std::max(0, std::min(n - 1, (int)(rmid / h)));
    const double tt = rmid / h - jm;
    const Cubic& cm = hc[al][jm];
    m->fref[al] = cm.x + tt * (cm.y + tt * (cm.z + tt * cm.w));
    for (int j = 0; j < n; ++j) {
      hs[al][j].x -= m->fref[al];
      const Cubic& q = hs[al][j];
      h32[(size_t)al * n + j] = make_float4((float)q.x, (float)q.y, (float)q.z, (float)q.w);
    }
  }
  MCK(cudaMemcpyAsync(e32, h32.data(), sizeof(float4) * h32.size(), cudaMemcpyHostToDevice, m->st));
  MCK(cudaStreamSynchronize(m->st));
  const double err = screen_bound_in(hs, h, dmax, lo, hi);
  if (!std::isfinite(err)) return mfail(m, VCSGC_ERR_NONFINITE, "non-finite embedding table");
  for (int x = 0; x < m->K; ++x)
    for (int y = 0; y < m->K; ++y) a.emb_off[x * m->K + y] = (float)(m->fref[y] - m->fref[x]);
  MCK(cudaDeviceGetAttribute(&a.n_sm, cudaDevAttrMultiProcessorCount, m->device));
  a.emb32 = e32;
  a.emb_n = n;
  a.emb_ih = (float)a.embed[0].inv_h;
  a.emb_lo = (float)lo;
  a.emb_hi = (float)hi;
  a.emb_err = (float)err;
  a.rf_q = (m->nx + a.qx - 1) / a.qx;
  a.rf_n = 2LL * m->nz * m->ny * a.qx * a.rf_q;
  MTRY(malloc_dev(m, &a.rf, (size_t)m->R * a.rf_n));
  return VCSGC_OK;
}

int init(Multi* m, const vcsgc_lattice* L, const uint8_t* types, const vcsgc_multi_tables* T, int R,
         const double* phi, const double* kappa, const double* Tk, const double* c0, const uint64_t* seed_r,
         const int32_t period[3], void* stream, int device) {
  if (!L || !types || !T || !phi || !kappa || !Tk || !c0 || !period || R < 1)
    return mfail(m, VCSGC_ERR_INVALID_ARG, "null argument or n_replicas < 1");
  if (L->kind != 0) return mfail(m, VCSGC_ERR_INVALID_ARG, "the multicomponent form needs a rigid lattice (kind 0)");
  if (T->K < 2 || T->K > MK_MAX) return mfail(m, VCSGC_ERR_INVALID_ARG, "K must be 2..4");
  if (T->nr < 2 || T->nrho < 2 || !(T->dr > 0) || !(T->drho > 0) || !(T->rc > 0))
    return mfail(m, VCSGC_ERR_INVALID_ARG, "bad table grid");
  m->K = T->K;
  m->R = R;
  m->nx = L->nx;
  m->ny = L->ny;
  m->nz = L->nz;
  m->a = L->a;
  m->rc = T->rc;
  if (m->nx < 1 || m->ny < 1 || m->nz < 1 || !(m->a > 0)) return mfail(m, VCSGC_ERR_INVALID_ARG, "bad lattice");
  m->N = 2LL * m->nx * m->ny * m->nz;
  if (m->N >= (1LL << 30)) return mfail(m, VCSGC_ERR_INVALID_ARG, "lattice too large");
  const int n3[3] = {m->nx, m->ny, m->nz};
  for (int q = 0; q < 3; ++q) {
    if (period[q] < 1 || n3[q] % period[q]) return mfail(m, VCSGC_ERR_INVALID_ARG, "period does not divide the lattice");
    if (n3[q] * m->a <= 2.0 * m->rc) return mfail(m, VCSGC_ERR_INVALID_ARG, "lattice edge not longer than 2 r_c");
    if (n3[q] > period[q] && period[q] * m->a <= 2.0 * m->rc)
      return mfail(m, VCSGC_ERR_SCHEDULE, "same-colour sublattice sites closer than 2 r_c");
  }
  if (device >= 0) MCK(cudaSetDevice(device));
  MCK(cudaGetDevice(&m->device));
  if (stream) {
    m->st = static_cast<cudaStream_t>(stream);
  } else {
    MCK(cudaStreamCreateWithFlags(&m->st, cudaStreamNonBlocking));
    m->own_stream = true;
  }
  MultiArgs& a = m->args;
  a.R = R;
  a.K = m->K;
  a.nx = m->nx;
  a.ny = m->ny;
  a.nz = m->nz;
  a.N = m->N;
  a.inv_n = 1.0 / (double)m->N;
  a.qx = period[0];
  a.qy = period[1];
  a.qz = period[2];
  a.nxq = m->nx / a.qx;
  a.nyq = m->ny / a.qy;
  a.nzq = m->nz / a.qz;
  a.n_colours = 2 * a.qx * a.qy * a.qz;
  a.D = a.nxq * a.nyq * a.nzq;
  m->steps_per_sweep = a.n_colours;
  // neighbour offsets h (half-lattice units, all even or all odd) with
  // (a/2)|h| < r_c, by |h|^2 then h; one shell per distinct |h|^2
  struct Off {
    int x, y, z, h2;
  };
  std::vector<Off> offs;
  const int H = (int)std::floor(2.0 * m->rc / m->a) + 1;
  for (int hx = -H; hx <= H; ++hx)
    for (int hy = -H; hy <= H; ++hy)
      for (int hz = -H; hz <= H; ++hz) {
        if ((hx & 1) != (hy & 1) || (hy & 1) != (hz & 1)) continue;
        const int h2 = hx * hx + hy * hy + hz * hz;
        if (h2 == 0 || 0.5 * m->a * std::sqrt((double)h2) >= m->rc) continue;
        offs.push_back({hx, hy, hz, h2});
      }
  std::sort(offs.begin(), offs.end(), [](const Off& p, const Off& q) {
    if (p.h2 != q.h2) return p.h2 < q.h2;
    if (p.x != q.x) return p.x < q.x;
    if (p.y != q.y) return p.y < q.y;
    return p.z < q.z;
  });
  if ((int)offs.size() > MK_MAX_OFF) return mfail(m, VCSGC_ERR_INVALID_ARG, "too many neighbours within r_c");
  std::vector<double> r_s;
  for (size_t k = 0; k < offs.size(); ++k) {
    if (k == 0 || offs[k].h2 != offs[k - 1].h2) r_s.push_back(0.5 * m->a * std::sqrt((double)offs[k].h2));
    a.off[k] = make_int4(offs[k].x, offs[k].y, offs[k].z, (int)r_s.size() - 1);
  }
  if ((int)r_s.size() > MK_MAX_SH) return mfail(m, VCSGC_ERR_INVALID_ARG, "too many neighbour shells within r_c");
  a.n_off = (int)offs.size();
  a.n_sh = (int)r_s.size();
  // tables: splines, then the shell values phi_ab(r_s), f_a(r_s)
  const int P = m->K * (m->K + 1) / 2;
  std::vector<Spline> sp_pair(P), sp_dens(m->K);
  for (int p = 0; p < P; ++p) {
    if (!T->pair[p]) return mfail(m, VCSGC_ERR_INVALID_ARG, "missing pair table");
    MTRY(make_spline(m, T->pair[p], T->dpair[p], T->nr, T->dr, sp_pair[p]));
  }
  for (int al = 0; al < m->K; ++al) {
    if (!T->dens[al] || !T->embed[al]) return mfail(m, VCSGC_ERR_INVALID_ARG, "missing density or embedding table");
    MTRY(make_spline(m, T->dens[al], T->ddens[al], T->nr, T->dr, sp_dens[al]));
    MTRY(make_spline(m, T->embed[al], T->dembed[al], T->nrho, T->drho, a.embed[al]));
  }
  Spline *d_pair = nullptr, *d_dens = nullptr;
  double *d_rs = nullptr, *V = nullptr, *Fd = nullptr;
  MTRY(malloc_dev(m, &d_pair, P));
  MTRY(malloc_dev(m, &d_dens, m->K));
  MTRY(malloc_dev(m, &d_rs, r_s.size()));
  MTRY(malloc_dev(m, &V, r_s.size() * m->K * m->K));
  MTRY(malloc_dev(m, &Fd, r_s.size() * m->K));
  MTRY(malloc_dev(m, &a.err, 1));
  MCK(cudaMemsetAsync(a.err, 0, sizeof(unsigned), m->st));
  MCK(cudaMemcpyAsync(d_pair, sp_pair.data(), sizeof(Spline) * P, cudaMemcpyHostToDevice, m->st));
  MCK(cudaMemcpyAsync(d_dens, sp_dens.data(), sizeof(Spline) * m->K, cudaMemcpyHostToDevice, m->st));
  MCK(cudaMemcpyAsync(d_rs, r_s.data(), sizeof(double) * r_s.size(), cudaMemcpyHostToDevice, m->st));
  launch_multi_shell_tables(d_pair, d_dens, m->K, d_rs, a.n_sh, V, Fd, a.err, m->st);
  MCK(cudaGetLastError());
  a.V = V;
  a.Fd = Fd;
  a.rcp_nxq = 1.0f / (float)a.nxq;
  a.rcp_nyq = 1.0f / (float)a.nyq;
  // fixed-point pair differences: the scale keeps 58 x 24 x max|dphi| < 2^62
  std::vector<double> hV(r_s.size() * m->K * m->K);
  MCK(cudaMemcpyAsync(hV.data(), V, sizeof(double) * hV.size(), cudaMemcpyDeviceToHost, m->st));
  std::vector<double> hFd(r_s.size() * m->K);
  MCK(cudaMemcpyAsync(hFd.data(), Fd, sizeof(double) * hFd.size(), cudaMemcpyDeviceToHost, m->st));
  MCK(cudaStreamSynchronize(m->st));
  MTRY(device_error(m));
  a.reembed = 0;
  for (int s = 0; s < a.n_sh; ++s)
    for (int al = 1; al < m->K; ++al)
      if (hFd[s * m->K + al] != hFd[s * m->K]) a.reembed = 1;
  double vmax = 0.0;
  for (double v : hV) vmax = std::max(vmax, std::fabs(v));
  if (!std::isfinite(vmax)) return mfail(m, VCSGC_ERR_NONFINITE, "non-finite pair table at a shell");
  // |phi_b - phi_a| <= 2 vmax; 58 x 24 x 2 vmax x 2^qbits < 2^62
  a.qbits = 52;
  while (a.qbits > 0 && 2.0 * vmax * 58.0 * 24.0 * std::ldexp(1.0, a.qbits) >= std::ldexp(1.0, 62)) --a.qbits;
  a.qscale = std::ldexp(1.0, -a.qbits);
  long long* Dq = nullptr;
  MTRY(malloc_dev(m, &Dq, (size_t)a.n_sh * m->K * m->K * m->K));
  launch_multi_fixed(V, a.n_sh, m->K, a.qbits, Dq, m->st);
  MCK(cudaGetLastError());
  a.Dq = Dq;
  a.bcc5 = a.n_off == MK_BCC5_N ? 1 : 0;
  for (int k = 0; k < a.n_off && a.bcc5; ++k) {
    const int code = mk_bcc5_code(k);
    if (a.off[k].x != (code & 15) - 4 || a.off[k].y != ((code >> 4) & 15) - 4 ||
        a.off[k].z != ((code >> 8) & 15) - 4 || a.off[k].w != code >> 12)
      a.bcc5 = 0;
  }
  // state
  MTRY(malloc_dev(m, &a.types, (size_t)R * m->N));
  MTRY(malloc_dev(m, &a.rho, (size_t)R * m->N));
  MRepParams* rp = nullptr;
  MTRY(malloc_dev(m, &rp, R));
  a.rp = rp;
  MTRY(malloc_dev(m, &a.rs, R));
  MTRY(malloc_dev(m, &a.acc, 3 * R));
  MTRY(malloc_dev(m, &a.pend, (size_t)R * a.D));
  m->n_part = multi_energy_blocks(m->N);
  MTRY(malloc_dev(m, &m->part, m->n_part));
  MCK(cudaMemsetAsync(a.acc, 0, sizeof(MStepAcc) * 3 * R, m->st));
  // fused form: one launch per colour step (no re-embedding, five-shell table)
  a.fused = (!a.reembed && a.bcc5) ? 1 : 0;
  MTRY(malloc_dev(m, &a.slot, (size_t)R * a.D));
  MCK(cudaMemsetAsync(a.slot, 0xFF, sizeof(int) * R * a.D, m->st));
  MTRY(malloc_dev(m, &a.nstart, (size_t)R * 2 * MK_MAX));
  MCK(cudaMemsetAsync(a.nstart, 0, sizeof(long long) * R * 2 * MK_MAX, m->st));
  MTRY(malloc_dev(m, &m->d_base, 1));
  MCK(cudaMemsetAsync(m->d_base, 0, sizeof(long long), m->st));
  a.base = m->d_base;
  a.qscale32 = (float)a.qscale;
  // screened form (re-embedding, five-shell table)
  // its commit indexes (accept, neighbour) items of all replicas in int:
  // every replica accepting every trial must stay below 2^31 items
  const bool items_fit = (long long)R * a.D * (MK_BCC5_N + 1) < (1LL << 31);
  a.screen = (a.reembed && a.bcc5 && R <= MK_SCREEN_MAX_R && items_fit) ? 1 : 0;
  if (a.screen) MTRY(screen_setup(m, hFd));
  MCK(cudaMemsetAsync(a.rs, 0, sizeof(MRepState) * R, m->st));
  m->h_rp.resize(R);
  const int S = m->K - 1;
  for (int r = 0; r < R; ++r) {
    const uint8_t* t = types + (long long)r * m->N;
    MTRY(load_replica(m, r, t, true));
    long long cnt[MK_MAX] = {0, 0, 0, 0};
    for (long long i = 0; i < m->N; ++i) cnt[t[i]]++;
    MRepParams& p = m->h_rp[r];
    p = MRepParams{};
    if (!(Tk[r] > 0)) return mfail(m, VCSGC_ERR_INVALID_ARG, "T must be > 0");
    p.beta = 1.0 / (KB_EV * Tk[r]);
    for (int al = 1; al < m->K; ++al) {
      const double ph = phi[(long long)r * S + al - 1], ka = kappa[(long long)r * S + al - 1];
      const double cc = c0[(long long)r * S + al - 1];
      p.phi[al] = ph;
      p.kappa_p[al] = ka * KB_EV * Tk[r] / (double)m->N;
      p.n0[al] = (double)m->N * (cc < 0.0 ? (double)cnt[al] / (double)m->N : cc);
      p.dmu0[al] = ph + 2.0 * p.kappa_p[al] * p.n0[al];
    }
    const uint64_t seed = seed_r ? seed_r[r] : (uint64_t)r + 1;
    p.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  }
  // without re-embedding every site has the density of site 0: the own
  // embedding change is a K x K table
  double* dF = nullptr;
  MTRY(malloc_dev(m, &dF, MK_MAX * MK_MAX));
  launch_multi_df(a, dF, m->st);
  MCK(cudaGetLastError());
  a.dF = dF;
  // float constants of the local screen: dF_ab + dmu0_b - dmu0_a, beta
  std::vector<double> hdF(MK_MAX * MK_MAX);
  MCK(cudaMemcpyAsync(hdF.data(), dF, sizeof(double) * m->K * m->K, cudaMemcpyDeviceToHost, m->st));
  MCK(cudaStreamSynchronize(m->st));
  for (int r = 0; r < R; ++r) {
    MRepParams& p = m->h_rp[r];
    p.beta32 = (float)p.beta;
    for (int x = 0; x < m->K; ++x)
      for (int y = 0; y < m->K; ++y) {
        p.c32[x * m->K + y] = (float)(hdF[x * m->K + y] + p.dmu0[y] - p.dmu0[x]);
        // the screened form's FP32 embedding tables are offset by fref
        const double off = a.screen ? m->fref[y] - m->fref[x] : 0.0;
        p.cmu32[x * m->K + y] = (float)(p.dmu0[y] - p.dmu0[x] + off);
      }
  }
  MCK(cudaMemcpyAsync(rp, m->h_rp.data(), sizeof(MRepParams) * R, cudaMemcpyHostToDevice, m->st));
  MCK(cudaStreamSynchronize(m->st));
  return VCSGC_OK;
}

Multi* as_multi(void* h) { return static_cast<Multi*>(h); }

}  // namespace
}  // namespace vcsgc

using namespace vcsgc;

extern "C" {

int vcsgc_multi_init(void** out, const vcsgc_lattice* lattice, const uint8_t* types, const vcsgc_multi_tables* tables,
                     int32_t n_replicas, const double* phi, const double* kappa, const double* T, const double* c0,
                     const uint64_t* seed_r, const int32_t period[3], void* stream, int32_t device) {
  VCSGC_TRACE("vcsgc_multi_init");
  if (!out) return VCSGC_ERR_INVALID_ARG;
  *out = nullptr;
  Multi* m = new (std::nothrow) Multi();
  if (!m) return VCSGC_ERR_NOMEM;
  const int rc = init(m, lattice, types, tables, n_replicas, phi, kappa, T, c0, seed_r, period, stream, device);
  if (rc != VCSGC_OK) {
    g_init_err = m->err;
    destroy(m);
    return rc;
  }
  *out = m;
  return VCSGC_OK;
}

int vcsgc_multi_steps(void* h, int64_t n) {
  VCSGC_TRACE("vcsgc_multi_steps");
  Multi* m = as_multi(h);
  if (!m || n < 0) return VCSGC_ERR_INVALID_ARG;
  MCK(cudaSetDevice(m->device));
  return run_steps(m, n);
}

int vcsgc_multi_sweep(void* h, int64_t n) {
  VCSGC_TRACE("vcsgc_multi_sweep");
  Multi* m = as_multi(h);
  if (!m || n < 0) return VCSGC_ERR_INVALID_ARG;
  MCK(cudaSetDevice(m->device));
  return run_steps(m, n * m->steps_per_sweep);
}

int vcsgc_multi_steps_per_sweep(void* h, int64_t* out) {
  Multi* m = as_multi(h);
  if (!m || !out) return VCSGC_ERR_INVALID_ARG;
  *out = m->steps_per_sweep;
  return VCSGC_OK;
}

int vcsgc_multi_observables(void* h, int32_t r, vcsgc_multi_obs* o) {
  VCSGC_TRACE("vcsgc_multi_observables");
  Multi* m = as_multi(h);
  if (!m || !o || r < 0 || r >= m->R) return VCSGC_ERR_INVALID_ARG;
  MCK(cudaSetDevice(m->device));
  MTRY(flush(m));
  MRepState s;
  MCK(cudaMemcpyAsync(&s, m->args.rs + r, sizeof(MRepState), cudaMemcpyDeviceToHost, m->st));
  MCK(cudaStreamSynchronize(m->st));
  MTRY(device_error(m));
  // the screened form does not track the energy (an accepted step would
  // need 118 FP64 embedding evaluations per flip): it is recomputed here
  if (m->args.screen) MTRY(energy_of(m, r, &s.energy));
  const MRepParams& p = m->h_rp[r];
  std::memset(o, 0, sizeof(*o));
  o->n_sites = m->N;
  o->K = m->K;
  o->energy = s.energy;
  o->energy_per_atom = s.energy / (double)m->N;
  o->steps = s.steps;
  o->trials = s.trials;
  o->local_accepts = s.local_acc;
  o->global_trials = s.global_trials;
  o->global_accepts = s.global_acc;
  o->flips = s.flips;
  o->near_ties = s.near_ties;
  o->stage1_accepts = s.s1_acc;
  o->acc_local = s.trials ? (double)s.local_acc / (double)s.trials : 0.0;
  o->acc_global = s.global_trials ? (double)s.global_acc / (double)s.global_trials : 0.0;
  o->sweeps = (double)s.trials / (double)m->N;
  for (int al = 0; al < m->K; ++al) {
    o->n[al] = s.cnt[al];
    o->c[al] = (double)s.cnt[al] / (double)m->N;
    o->mean_c[al] = s.steps ? s.sum_c[al] / (double)s.steps : o->c[al];
    o->var_c[al] = s.steps ? std::max(0.0, s.sum_c2[al] / (double)s.steps - o->mean_c[al] * o->mean_c[al]) : 0.0;
    o->kappa_p[al] = p.kappa_p[al];
    o->dmu0[al] = p.dmu0[al];
    o->dmu_est[al] = al ? p.phi[al] + 2.0 * p.kappa_p[al] * (double)m->N * o->mean_c[al] : 0.0;
  }
  return VCSGC_OK;
}

int vcsgc_multi_get_types(void* h, int32_t r, uint8_t* out) {
  VCSGC_TRACE("vcsgc_multi_get_types");
  Multi* m = as_multi(h);
  if (!m || !out || r < 0 || r >= m->R) return VCSGC_ERR_INVALID_ARG;
  MCK(cudaSetDevice(m->device));
  MTRY(flush(m));
  MCK(cudaMemcpyAsync(out, m->args.types + (long long)r * m->N, m->N, cudaMemcpyDeviceToHost, m->st));
  MCK(cudaStreamSynchronize(m->st));
  return VCSGC_OK;
}

int vcsgc_multi_set_types(void* h, int32_t r, const uint8_t* in) {
  VCSGC_TRACE("vcsgc_multi_set_types");
  Multi* m = as_multi(h);
  if (!m || !in || r < 0 || r >= m->R) return VCSGC_ERR_INVALID_ARG;
  MCK(cudaSetDevice(m->device));
  return load_replica(m, r, in, false);
}

int vcsgc_multi_delta_e(void* h, int32_t r, const int64_t* sites, const uint8_t* to, int64_t n, double* out) {
  Multi* m = as_multi(h);
  if (!m || r < 0 || r >= m->R || n < 0 || (n > 0 && (!sites || !to || !out)) || n > (1LL << 30))
    return VCSGC_ERR_INVALID_ARG;
  for (int64_t q = 0; q < n; ++q)
    if (sites[q] < 0 || sites[q] >= m->N || to[q] >= m->K) return mfail(m, VCSGC_ERR_INVALID_ARG, "site or species out of range");
  if (n == 0) return VCSGC_OK;
  MCK(cudaSetDevice(m->device));
  if (n > m->buf_n) {
    MTRY(malloc_dev(m, &m->d_sites, n));
    MTRY(malloc_dev(m, &m->d_to, n));
    MTRY(malloc_dev(m, &m->d_out, n));
    m->buf_n = n;
  }
  MTRY(flush(m));
  MCK(cudaMemcpyAsync(m->d_sites, sites, sizeof(long long) * n, cudaMemcpyHostToDevice, m->st));
  MCK(cudaMemcpyAsync(m->d_to, to, n, cudaMemcpyHostToDevice, m->st));
  launch_multi_delta_e(m->args, r, m->d_sites, m->d_to, (int)n, m->d_out, m->st);
  MCK(cudaGetLastError());
  MCK(cudaMemcpyAsync(out, m->d_out, sizeof(double) * n, cudaMemcpyDeviceToHost, m->st));
  MCK(cudaStreamSynchronize(m->st));
  return device_error(m);
}

int vcsgc_multi_energy(void* h, int32_t r, double* out) {
  Multi* m = as_multi(h);
  if (!m || !out || r < 0 || r >= m->R) return VCSGC_ERR_INVALID_ARG;
  MCK(cudaSetDevice(m->device));
  MTRY(flush(m));
  return energy_of(m, r, out);
}

int vcsgc_multi_set_surrogate(void* h, void* mlp) {
  VCSGC_TRACE("vcsgc_multi_set_surrogate");
  Multi* m = as_multi(h);
  if (!m) return VCSGC_ERR_INVALID_ARG;
  MCK(cudaSetDevice(m->device));
  MultiArgs& a = m->args;
  if (!mlp) {
    MCK(cudaStreamSynchronize(m->st));
    a.da = 0;
    drop_graph(m);
    return VCSGC_OK;
  }
  if (m->K != 2 || !a.screen)
    return mfail(m, VCSGC_ERR_STATE,
                 "delayed acceptance needs K = 2 with species-dependent densities on the five-shell table");
  MlpBuf src{};
  if (!mlp_object_buffers(mlp, &src)) return VCSGC_ERR_INVALID_ARG;
  if (!m->sur.w1f) {
    MTRY(malloc_dev(m, &m->sur.w1f, MLP_W1F));
    MTRY(malloc_dev(m, &m->sur.w2f, MLP_W2F));
    MTRY(malloc_dev(m, &m->sur.w2tf, MLP_W2F));
    MTRY(malloc_dev(m, &m->sur.vec, MLP_VEC));
  }
  if (!a.nbc) {
    MTRY(malloc_dev(m, &a.nbc, (size_t)m->R * a.rf_n));
    m->nbc_stale = true;
  }
  // the surrogate's own stream may still be writing its fragments
  MCK(cudaStreamSynchronize(mlp_object_stream(mlp)));
  MCK(cudaMemcpyAsync(m->sur.w1f, src.w1f, sizeof(uint2) * MLP_W1F, cudaMemcpyDeviceToDevice, m->st));
  MCK(cudaMemcpyAsync(m->sur.w2f, src.w2f, sizeof(uint2) * MLP_W2F, cudaMemcpyDeviceToDevice, m->st));
  MCK(cudaMemcpyAsync(m->sur.w2tf, src.w2tf, sizeof(uint2) * MLP_W2F, cudaMemcpyDeviceToDevice, m->st));
  MCK(cudaMemcpyAsync(m->sur.vec, src.vec, sizeof(float) * MLP_VEC, cudaMemcpyDeviceToDevice, m->st));
  MCK(cudaStreamSynchronize(m->st));
  a.mlp = mlp_view(m->sur);
  a.da = 1;
  drop_graph(m);  // the captured steps hold the arguments by value
  return VCSGC_OK;
}

int vcsgc_multi_features(void* h, float* d_X, float* d_Y) {
  VCSGC_TRACE("vcsgc_multi_features");
  Multi* m = as_multi(h);
  if (!m || !d_X || !d_Y) return VCSGC_ERR_INVALID_ARG;
  MCK(cudaSetDevice(m->device));
  MultiArgs& a = m->args;
  if (m->K != 2 || !a.screen)
    return mfail(m, VCSGC_ERR_STATE,
                 "features need K = 2 with species-dependent densities on the five-shell table");
  if (!a.nbc) {
    MTRY(malloc_dev(m, &a.nbc, (size_t)m->R * a.rf_n));
    m->nbc_stale = true;
  }
  MTRY(nbc_fresh(m));
  launch_multi_features(a, d_X, d_Y, m->st);
  MCK(cudaGetLastError());
  MCK(cudaStreamSynchronize(m->st));
  return device_error(m);
}

const char* vcsgc_multi_last_error(void* h) {
  Multi* m = as_multi(h);
  return m ? m->err.c_str() : g_init_err.c_str();
}

void vcsgc_multi_free(void* h) { destroy(as_multi(h)); }

}  // extern "C"

// ---- host-side access for a binary context that runs its colour steps
//      through a two-species multicomponent object (multi_host.h)
namespace vcsgc {

int multi_get_state(void* h, int r, MRepState* out) {
  Multi* m = as_multi(h);
  if (!m || !out || r < 0 || r >= m->R) return VCSGC_ERR_INVALID_ARG;
  MCK(cudaSetDevice(m->device));
  MTRY(flush(m));
  MCK(cudaMemcpyAsync(out, m->args.rs + r, sizeof(MRepState), cudaMemcpyDeviceToHost, m->st));
  MCK(cudaStreamSynchronize(m->st));
  return device_error(m);
}

int multi_set_state(void* h, int r, const MRepState* in) {
  Multi* m = as_multi(h);
  if (!m || !in || r < 0 || r >= m->R || m->args.fused) return VCSGC_ERR_INVALID_ARG;
  MCK(cudaSetDevice(m->device));
  MCK(cudaMemcpyAsync(m->args.rs + r, in, sizeof(MRepState), cudaMemcpyHostToDevice, m->st));
  MCK(cudaStreamSynchronize(m->st));
  // screened form: the replicas step together from the device base
  if (m->args.screen) {
    m->h_base = in->step;
    m->acc_stale = true;
  }
  return VCSGC_OK;
}

int multi_get_rho(void* h, int r, double* out) {
  Multi* m = as_multi(h);
  if (!m || !out || r < 0 || r >= m->R) return VCSGC_ERR_INVALID_ARG;
  MCK(cudaSetDevice(m->device));
  MTRY(flush(m));
  MCK(cudaMemcpyAsync(out, m->args.rho + (long long)r * m->N, sizeof(double) * m->N, cudaMemcpyDeviceToHost, m->st));
  MCK(cudaStreamSynchronize(m->st));
  return VCSGC_OK;
}

bool multi_screened(void* h) {
  Multi* m = as_multi(h);
  return m && m->args.screen;
}

const uint8_t* multi_types_device(void* h, int r) {
  Multi* m = as_multi(h);
  if (!m || r < 0 || r >= m->R || flush(m) != VCSGC_OK) return nullptr;
  return m->args.types + (long long)r * m->N;
}

}  // namespace vcsgc
