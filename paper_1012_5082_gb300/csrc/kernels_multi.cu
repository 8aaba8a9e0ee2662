// Multicomponent colour step (K <= 4 species, rigid BCC lattice, period-q
// sublattice schedule).  The paper works the method out for a binary alloy
// and notes that the generalisation to more species is straightforward
// (Sec. II); the form built here keeps one variance constraint per solute
// species alpha = 1..K-1:
//   pi_V ~ exp{-beta [U + sum_alpha (phi_alpha n_alpha + kappa_p,alpha n_alpha^2)]}.
// A trial at site i of species a proposes species b, uniform among the K-1
// others.  Local stage (Eq. trans_vcsgc_par1 per solute):
//   min{1, exp[-beta (dE_i + dmu0_b - dmu0_a)]},  dmu0_0 = 0;
// global stage (Eq. trans_vcsgc_par2 per solute):
//   min{1, exp[-beta sum_alpha kappa_p,alpha dn_alpha (dn_alpha + 2 (n_alpha - n0_alpha))]}.
//
// One thread per trial.  dE on the rigid lattice: the pair part from the
// per-shell neighbour counts by species (one 64-bit word per species, 8 bits
// per shell) against the shell table phi_ab(r_s) staged in shared memory; the
// own embedding change F_b(rho_i) - F_a(rho_i); and, where the densities
// differ between species, the re-embedding of every neighbour j,
// F_{t_j}(rho_j + f_b(r_s) - f_a(r_s)) - F_{t_j}(rho_j).  Two launches per
// colour step: propose (local stage, compaction of the accepts, per-solute
// dn by warp reductions; the last block of each replica takes the global
// decision) and commit (species and density scatter of an accepted step).
// With re-embedding on the five-shell table the propose is FP32-screened
// (below) and the commit runs one thread per (accept, neighbour); without
// re-embedding one fused launch per step carries both (k_multi_fused).
#include "multi.cuh"

namespace vcsgc {

__host__ __device__ __forceinline__ int multi_tri(int K, int a, int b) {
  if (a > b) {
    const int q = a;
    a = b;
    b = q;
  }
  return a * K - a * (a - 1) / 2 + (b - a);
}


__global__ void k_multi_shell_tables(const Spline* pair, const Spline* dens, int K, const double* r_s, int n_sh,
                                     double* V, double* Fd, unsigned* err) {
  const int nv = n_sh * K * K;
  for (int q = threadIdx.x; q < nv; q += blockDim.x) {
    const int s = q / (K * K), a = (q / K) % K, b = q % K;
    V[q] = spline_val(pair[multi_tri(K, a, b)], r_s[s], err);
  }
  for (int q = threadIdx.x; q < n_sh * K; q += blockDim.x) Fd[q] = spline_val(dens[q % K], r_s[q / K], err);
}

void launch_multi_shell_tables(const Spline* pair, const Spline* dens, int K, const double* r_s, int n_sh,
                               double* V, double* Fd, unsigned* err, cudaStream_t st) {
  k_multi_shell_tables<<<1, 128, 0, st>>>(pair, dens, K, r_s, n_sh, V, Fd, err);
}

__global__ void k_multi_fixed(const double* V, int n_sh, int K, int qbits, long long* Dq) {
  const int n = n_sh * K * K * K;
  const double sc = ldexp(1.0, qbits);
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const int be = q % K, b = (q / K) % K, a = (q / (K * K)) % K, s = q / (K * K * K);
    Dq[q] = llrint((V[(s * K + b) * K + be] - V[(s * K + a) * K + be]) * sc);
  }
}

void launch_multi_fixed(const double* V, int n_sh, int K, int qbits, long long* Dq, cudaStream_t st) {
  k_multi_fixed<<<1, 256, 0, st>>>(V, n_sh, K, qbits, Dq);
}

// rho_i = sum_j f_{t_j}(r_ij)
__global__ void k_multi_rho(MultiArgs a, int r0) {
  const int r = r0 + blockIdx.y;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  const uint8_t* ty = a.types + (long long)r * a.N;
  double rho = 0.0;
  for (int k = 0; k < a.n_off; ++k) {
    const int4 h = a.off[k];
    rho += a.Fd[h.w * a.K + ty[multi_nbr(a, (int)i, h)]];
  }
  a.rho[(long long)r * a.N + i] = rho;
  if (a.rf) {
    const float r32 = (float)rho;
    const int3 h = multi_half(a, (int)i);
    const int b = (int)(i & 1);
    a.rf[(long long)r * a.rf_n + multi_rfi(a, (h.x - b) >> 1, (h.y - b) >> 1, (h.z - b) >> 1, b)] =
        make_float2(r32, emb32_val(a, ty[i], r32));
  }
}

void launch_multi_rho(const MultiArgs& a, int r0, int nrep, cudaStream_t st) {
  const dim3 grid((unsigned)((a.N + 255) / 256), (unsigned)nrep);
  k_multi_rho<<<grid, 256, 0, st>>>(a, r0);
}

// E = sum_i [1/2 sum_j phi_{t_i t_j}(r_ij) + F_{t_i}(rho_i)], block partials
constexpr int MK_EBLOCK = 256;

int multi_energy_blocks(long long N) { return (int)((N + MK_EBLOCK - 1) / MK_EBLOCK); }

__global__ void __launch_bounds__(MK_EBLOCK) k_multi_energy(MultiArgs a, int r0, double* part) {
  const int r = r0 + blockIdx.y;
  const long long i = (long long)blockIdx.x * MK_EBLOCK + threadIdx.x;
  double e = 0.0;
  if (i < a.N) {
    const uint8_t* ty = a.types + (long long)r * a.N;
    const int ti = ty[i];
    double pair = 0.0;
    for (int k = 0; k < a.n_off; ++k) {
      const int4 h = a.off[k];
      pair += a.V[(h.w * a.K + ti) * a.K + ty[multi_nbr(a, (int)i, h)]];
    }
    e = 0.5 * pair + spline_val(a.embed[ti], a.rho[(long long)r * a.N + i], a.err);
  }
  __shared__ double sh[MK_EBLOCK / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < MK_EBLOCK / 32; ++w) t += sh[w];
    part[(long long)blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

void launch_multi_energy(const MultiArgs& a, int r0, int nrep, double* part, cudaStream_t st) {
  const dim3 grid((unsigned)multi_energy_blocks(a.N), (unsigned)nrep);
  k_multi_energy<<<grid, MK_EBLOCK, 0, st>>>(a, r0, part);
}

// dE of site i (replica r) going from species ta to tb; sV, sFd: the shell
// tables (shared or global).  The neighbours are visited in chunks of 8:
// the chunk's index arithmetic and loads are issued before any of its sums,
// so up to 8 L2 reads per thread are in flight at once.  Per-shell counts by
// species sit in one 64-bit word per species (8 bits per shell).
constexpr int MK_CHUNK = 8;

template <bool REEMBED>
__device__ double multi_de(const MultiArgs& a, const double* sV, const double* sFd, int r, int i, int ta, int tb) {
  const uint8_t* ty = a.types + (long long)r * a.N;
  const double* rho = a.rho + (long long)r * a.N;
  const int K = a.K;
  const int3 p = multi_half(a, i);
  unsigned long long c0 = 0ull, c1 = 0ull, c2 = 0ull, c3 = 0ull;
  double re = 0.0;
  for (int k0 = 0; k0 < a.n_off; k0 += MK_CHUNK) {
    int tj[MK_CHUNK];
    double rj[MK_CHUNK];
#pragma unroll
    for (int u = 0; u < MK_CHUNK; ++u) {
      const int k = k0 + u;
      tj[u] = 0;
      rj[u] = 0.0;
      if (k < a.n_off) {
        const int j = multi_nbr_at(a, p, a.off[k]);
        tj[u] = ty[j];
        if constexpr (REEMBED) rj[u] = rho[j];
      }
    }
#pragma unroll
    for (int u = 0; u < MK_CHUNK; ++u) {
      const int k = k0 + u;
      if (k < a.n_off) {
        const int s = a.off[k].w;
        const unsigned long long inc = 1ull << (8 * s);
        c0 += tj[u] == 0 ? inc : 0ull;
        c1 += tj[u] == 1 ? inc : 0ull;
        c2 += tj[u] == 2 ? inc : 0ull;
        c3 += tj[u] == 3 ? inc : 0ull;
        if constexpr (REEMBED) {
          const double dfs = sFd[s * K + tb] - sFd[s * K + ta];
          re += spline_val(a.embed[tj[u]], rj[u] + dfs, a.err) - spline_val(a.embed[tj[u]], rj[u], a.err);
        }
      }
    }
  }
  double pair = 0.0;
  for (int s = 0; s < a.n_sh; ++s) {
    const double* Vb = sV + (s * K + tb) * K;
    const double* Va = sV + (s * K + ta) * K;
    const int sh = 8 * s;
    pair += (double)((c0 >> sh) & 255ull) * (Vb[0] - Va[0]);
    pair += (double)((c1 >> sh) & 255ull) * (Vb[1] - Va[1]);
    if (K > 2) pair += (double)((c2 >> sh) & 255ull) * (Vb[2] - Va[2]);
    if (K > 3) pair += (double)((c3 >> sh) & 255ull) * (Vb[3] - Va[3]);
  }
  const double ri = rho[i];
  const double own = spline_val(a.embed[tb], ri, a.err) - spline_val(a.embed[ta], ri, a.err);
  return pair + own + re;
}

// The same dE with the compile-time five-shell table, basis B of the trial
// site in cell (cx, cy, cz): the wrapped x, y, z offsets of the cells -2..2
// are computed once, every neighbour index is then three adds, and the
// per-shell counts sit in one 32-bit word per shell (8 bits per species).
// Without re-embedding the density is the same at every site and the own
// embedding change comes from the table sDF[a K + b].
__device__ __forceinline__ int mk_wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// n / d for 0 <= n < 2^22 from the float reciprocal, corrected to the exact
// quotient
__device__ __forceinline__ int mk_div(int n, int d, float rcp) {
  int q = __float2int_rz(__int2float_rn(n) * rcp);
  const int rr = n - q * d;
  q += rr < 0 ? -1 : (rr >= d ? 1 : 0);
  return q;
}

template <int B, bool REEMBED>
__device__ double multi_de_bcc5(const MultiArgs& a, const long long* sDq, const double* sFd, const double* sDF, int r,
                                int i, int cx, int cy, int cz, int ta, int tb) {
  const uint8_t* ty = a.types + (long long)r * a.N;
  const double* rho = a.rho + (long long)r * a.N;
  const int K = a.K;
  int xo[5], yo[5], zo[5];
#pragma unroll
  for (int d = -2; d <= 2; ++d) {
    xo[d + 2] = 2 * mk_wrap(cx + d, a.nx);
    yo[d + 2] = 2 * a.nx * mk_wrap(cy + d, a.ny);
    zo[d + 2] = 2 * a.nx * a.ny * mk_wrap(cz + d, a.nz);
  }
  unsigned cnt[5] = {0u, 0u, 0u, 0u, 0u};
  double re = 0.0;
  // without re-embedding all 58 species loads are issued at once; with it,
  // chunks of 8 (each also loads a density)
  constexpr int CH = REEMBED ? MK_CHUNK : MK_BCC5_N;
#pragma unroll
  for (int k0 = 0; k0 < MK_BCC5_N; k0 += CH) {
    int tj[CH];
    double rj[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      if (k0 + u < MK_BCC5_N) {
        const int code = mk_bcc5_code(k0 + u);
        const int hx = (code & 15) - 4, hy = ((code >> 4) & 15) - 4, hz = ((code >> 8) & 15) - 4;
        const int bb = B ^ (hx & 1);
        const int j = zo[((B + hz - bb) >> 1) + 2] + yo[((B + hy - bb) >> 1) + 2] + xo[((B + hx - bb) >> 1) + 2] + bb;
        tj[u] = ty[j];
        if constexpr (REEMBED) rj[u] = rho[j];
      }
    }
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      if (k0 + u < MK_BCC5_N) {
        const int s = mk_bcc5_code(k0 + u) >> 12;
        cnt[s] += 1u << (8 * tj[u]);
        if constexpr (REEMBED) {
          const double dfs = sFd[s * K + tb] - sFd[s * K + ta];
          re += spline_val(a.embed[tj[u]], rj[u] + dfs, a.err) - spline_val(a.embed[tj[u]], rj[u], a.err);
        }
      }
    }
  }
  // pair part: integer counts times the fixed-point differences, exact in
  // 64 bits; one conversion to FP64 at the end
  long long pq = 0;
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const long long* D = sDq + ((s * K + ta) * K + tb) * K;
    for (int be = 0; be < K; ++be) pq += (long long)((cnt[s] >> (8 * be)) & 255u) * D[be];
  }
  const double pair = (double)pq * a.qscale;
  double own;
  if constexpr (REEMBED) {
    const double ri = rho[i];
    own = spline_val(a.embed[tb], ri, a.err) - spline_val(a.embed[ta], ri, a.err);
  } else {
    own = sDF[ta * K + tb];
  }
  return pair + own + re;
}

// ------------------------------------------------------ screened form
// With re-embedding a trial's dE holds 2 x 58 + 2 embedding evaluations,
// which in FP64 (a small share of GB300's arithmetic) bound the step.  The
// local decision is taken instead on an FP32 dE whose distance from the
// FP64 dE has a proven bound: per evaluation emb_err (coefficient rounding,
// Horner rounding, and the argument rounding of rho, f_b(r_s) - f_a(r_s)
// and x / h times the slope), plus 2^-18 of the sum of |terms| for the 58
// float additions and 2^-21 of the sizes of the final sums.  A trial whose
// screen cannot decide, or whose argument leaves [emb_lo, emb_hi], gets its
// dE in FP64 from the whole warp: 32 lanes share its 58 neighbours and two
// own-site terms.  Every decision is therefore the one the FP64 dE takes.

// FP32 dE of site i (cell (cx, cy, cz)) from species ta to tb without the
// chemical-potential term; *err bounds its distance from the FP64 dE, *pq
// is the exact fixed-point pair part, *in is false when an argument left
// the bounded range.  sDfs[(s K + a) K + b] = f_b(r_s) - f_a(r_s) as
// floats; sw: this block's [30][MK_BLOCK] scratch for the wrapped cell
// offsets of the thread's site (x, y, z for cells -2..2), as species
// indices and as indices of the per-site floats; scode: the block's
// neighbour descriptors.  The neighbours are visited
// shell by shell, kScreenIlp at a time (loads in flight per thread against
// registers; a colour step of 64,000 trials gives about 13 warps per SM).

// descriptor of neighbour k of a basis-B site: cell indices (0..4 for
// -2..2) in bits 0-2, 3-5, 6-8, the neighbour's basis in bit 9 and its
// shell from bit 10
template <int B>
__host__ __device__ constexpr int mk_bcc5_desc(int k) {
  return (((B + ((mk_bcc5_code(k) & 15) - 4) - (B ^ (((mk_bcc5_code(k) & 15) - 4) & 1))) >> 1) + 2) |
         ((((B + (((mk_bcc5_code(k) >> 4) & 15) - 4) - (B ^ (((mk_bcc5_code(k) & 15) - 4) & 1))) >> 1) + 2) << 3) |
         ((((B + (((mk_bcc5_code(k) >> 8) & 15) - 4) - (B ^ (((mk_bcc5_code(k) & 15) - 4) & 1))) >> 1) + 2) << 6) |
         ((B ^ (((mk_bcc5_code(k) & 15) - 4) & 1)) << 9) | ((mk_bcc5_code(k) >> 12) << 10);
}

// first neighbour of shell s in the five-shell order (8, 6, 12, 24, 8 sites)
__host__ __device__ constexpr int mk_shell0(int s) {
  return s == 0 ? 0 : (s == 1 ? 8 : (s == 2 ? 14 : (s == 3 ? 26 : (s == 4 ? 50 : MK_BCC5_N))));
}

constexpr int kScreenIlp = 12;  // 125 registers, no spills; 4, 8, 12 measured within 3 %

__device__ float multi_screen_bcc5(const MultiArgs& a, const long long* sDq, const float* sDfs, int* sw,
                                   const int* scode, int r, int i, int cx, int cy, int cz, int ta, int tb,
                                   long long* pq_out, float* err, bool* in) {
  const uint8_t* ty = a.types + (long long)r * a.N;
  const float2* rf = a.rf + (long long)r * a.rf_n;
  const int K = a.K;
  const int tid = threadIdx.x;
  // wrapped offsets of cells -2..2: species index (sw[0..14]) and the
  // per-site floats' index (sw[15..29]); rplane: the basis-1 half of the latter
  const int rrow = a.qx * a.rf_q;
  const int rplane = a.nz * a.ny * rrow;
#pragma unroll
  for (int d = -2; d <= 2; ++d) {
    const int X = mk_wrap(cx + d, a.nx), xq = X / a.qx;
    sw[(d + 2) * MK_BLOCK + tid] = 2 * X;
    sw[(d + 7) * MK_BLOCK + tid] = 2 * a.nx * mk_wrap(cy + d, a.ny);
    sw[(d + 12) * MK_BLOCK + tid] = 2 * a.nx * a.ny * mk_wrap(cz + d, a.nz);
    sw[(d + 17) * MK_BLOCK + tid] = (X - xq * a.qx) * a.rf_q + xq;
    sw[(d + 22) * MK_BLOCK + tid] = rrow * mk_wrap(cy + d, a.ny);
    sw[(d + 27) * MK_BLOCK + tid] = rrow * a.ny * mk_wrap(cz + d, a.nz);
  }
  const float2 ri = rf[sw[17 * MK_BLOCK + tid] + sw[22 * MK_BLOCK + tid] + sw[27 * MK_BLOCK + tid] + (i & 1) * rplane];
  unsigned cnt[5];
  float re = 0.0f, ab = 0.0f;
  bool ok = true;
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const float df = sDfs[(s * K + ta) * K + tb];
    unsigned c = 0u;
#pragma unroll kScreenIlp
    for (int k = mk_shell0(s); k < mk_shell0(s + 1); ++k) {
      const int dc = scode[k];
      const int ix = dc & 7, iy = (dc >> 3) & 7, iz = (dc >> 6) & 7, bb = (dc >> 9) & 1;
      const int j = sw[ix * MK_BLOCK + tid] + sw[(5 + iy) * MK_BLOCK + tid] + sw[(10 + iz) * MK_BLOCK + tid] + bb;
      const int jr = sw[(15 + ix) * MK_BLOCK + tid] + sw[(20 + iy) * MK_BLOCK + tid] + sw[(25 + iz) * MK_BLOCK + tid] +
                     (bb ? rplane : 0);
      const int t = ty[j];
      const float2 v = rf[jr];
      c += 1u << (8 * t);
      const float x1 = v.x + df;
      ok &= emb32_in(a, v.x) & emb32_in(a, x1);
      const float d = emb32_val(a, t, x1) - v.y;
      re += d;
      ab += fabsf(d);
    }
    cnt[s] = c;
  }
  long long pq = 0;
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const long long* D = sDq + ((s * K + ta) * K + tb) * K;
    for (int be = 0; be < K; ++be) pq += (long long)((cnt[s] >> (8 * be)) & 255u) * D[be];
  }
  ok &= emb32_in(a, ri.x);
  const float own = emb32_val(a, tb, ri.x) - ri.y;
  const float pair = __ll2float_rn(pq) * a.qscale32;
  *pq_out = pq;
  *in = ok;
  *err = fmaf((float)(2 * MK_BCC5_N + 2), a.emb_err,
              fmaf(3.814697265625e-06f, ab, 4.76837158203125e-07f * (fabsf(pair) + fabsf(own) + fabsf(re))));
  return (pair + own) + re;
}

// The same FP32 dE by a group of MK_GROUP lanes of one warp (delayed
// acceptance, where only the block's stage-1 passes need it): lane gl of
// the group takes neighbours gl, gl + MK_GROUP, ... of the five-shell table
// and lane 0 the own-site term; the partial sums are combined by shuffles
// inside the group, so every lane of the group returns the trial's values.
// The partial sums change the order of the float additions only: at most 7
// sequential and 3 pairwise steps, well inside the 2^-18 sum(|terms|) of
// the bound.  gw: the group's [30] scratch of wrapped cell offsets (the
// layout of multi_screen_bcc5's sw); has: the group holds a trial.  Must be
// called by all 32 lanes.
constexpr int MK_GROUP = 8;

__device__ float multi_screen_group(const MultiArgs& a, const long long* sDq, const float* sDfs, int* gw,
                                    const int* scode, int r, int i, int cx, int cy, int cz, int ta, int tb, int gl,
                                    bool has, long long* pq_out, float* err, bool* in) {
  const uint8_t* ty = a.types + (long long)r * a.N;
  const float2* rf = a.rf + (long long)r * a.rf_n;
  const int K = a.K;
  const int rrow = a.qx * a.rf_q;
  const int rplane = a.nz * a.ny * rrow;
  for (int q = gl; has && q < 5; q += MK_GROUP) {
    const int dd = q - 2;
    const int X = mk_wrap(cx + dd, a.nx), xq = X / a.qx;
    const int Y = mk_wrap(cy + dd, a.ny), Z = mk_wrap(cz + dd, a.nz);
    gw[q] = 2 * X;
    gw[5 + q] = 2 * a.nx * Y;
    gw[10 + q] = 2 * a.nx * a.ny * Z;
    gw[15 + q] = (X - xq * a.qx) * a.rf_q + xq;
    gw[20 + q] = rrow * Y;
    gw[25 + q] = rrow * a.ny * Z;
  }
  __syncwarp();
  long long pq = 0;
  float re = 0.0f, ab = 0.0f, own = 0.0f;
  bool ok = true;
  if (has) {
    const float* Df = sDfs + (ta * K + tb);
    const long long* Dq = sDq + (ta * K + tb) * K;
#pragma unroll
    for (int m = 0; m < (MK_BCC5_N + MK_GROUP - 1) / MK_GROUP; ++m) {
      const int k = gl + MK_GROUP * m;
      if (k < MK_BCC5_N) {
        const int dc = scode[k];
        const int ix = dc & 7, iy = (dc >> 3) & 7, iz = (dc >> 6) & 7, bb = (dc >> 9) & 1, sh = dc >> 10;
        const int j = gw[ix] + gw[5 + iy] + gw[10 + iz] + bb;
        const int jr = gw[15 + ix] + gw[20 + iy] + gw[25 + iz] + (bb ? rplane : 0);
        const int t = ty[j];
        const float2 v = rf[jr];
        pq += Dq[sh * K * K * K + t];
        const float x1 = v.x + Df[sh * K * K];
        ok &= emb32_in(a, v.x) & emb32_in(a, x1);
        const float d = emb32_val(a, t, x1) - v.y;
        re += d;
        ab += fabsf(d);
      }
    }
    if (gl == 0) {
      const float2 ri = rf[gw[17] + gw[22] + gw[27] + (i & 1) * rplane];
      ok &= emb32_in(a, ri.x);
      own = emb32_val(a, tb, ri.x) - ri.y;
    }
  }
#pragma unroll
  for (int o = MK_GROUP / 2; o > 0; o >>= 1) {
    pq += __shfl_xor_sync(0xffffffffu, pq, o);
    re += __shfl_xor_sync(0xffffffffu, re, o);
    ab += __shfl_xor_sync(0xffffffffu, ab, o);
    own += __shfl_xor_sync(0xffffffffu, own, o);
  }
  const unsigned bad = __ballot_sync(0xffffffffu, !ok);
  const int lane = threadIdx.x & 31;
  ok = ((bad >> (lane & ~(MK_GROUP - 1))) & ((1u << MK_GROUP) - 1u)) == 0u;
  const float pair = __ll2float_rn(pq) * a.qscale32;
  *pq_out = pq;
  *in = ok;
  *err = fmaf((float)(2 * MK_BCC5_N + 2), a.emb_err,
              fmaf(3.814697265625e-06f, ab, 4.76837158203125e-07f * (fabsf(pair) + fabsf(own) + fabsf(re))));
  return (pair + own) + re;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ long long warp_sum(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Lane's share of the FP64 embedding part of the dE of site i from ta to tb
// (58 re-embeddings and the own-site change) on the compile-time five-shell
// table, for a warp that takes one trial the FP32 screen left open: lane l
// takes neighbours l and l + 32 (or, for l + 32 = 58 and 59, the own-site
// terms), in that order; warp_sum adds the lanes.  The neighbours come from the block's
// descriptors (scode, basis of site i) and fw, this warp's [15] scratch of
// wrapped cell offsets (species indices); both neighbours' species and
// densities load at once, then all four cubics.  Must be called by all 32
// lanes with the same i.
__device__ double multi_emb_warp5(const MultiArgs& a, const double* sFd, const int* scode, int* fw, int r, int i,
                                  int ta, int tb, int lane) {
  const uint8_t* ty = a.types + (long long)r * a.N;
  const double* rho = a.rho + (long long)r * a.N;
  const int K = a.K;
  const int cell = i >> 1, nxy = a.nx * a.ny;
  const int cz = cell / nxy, cy = (cell - cz * nxy) / a.nx, cx = cell - cz * nxy - cy * a.nx;
  if (lane < 5) {
    const int dd = lane - 2;
    fw[lane] = 2 * mk_wrap(cx + dd, a.nx);
    fw[5 + lane] = 2 * a.nx * mk_wrap(cy + dd, a.ny);
    fw[10 + lane] = 2 * nxy * mk_wrap(cz + dd, a.nz);
  }
  __syncwarp();
  int jj[2], tj[2], sh[2];
  double rj[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int k = lane + 32 * u;
    jj[u] = i;
    sh[u] = 0;
    if (k < MK_BCC5_N) {
      const int dc = scode[k];
      jj[u] = fw[dc & 7] + fw[5 + ((dc >> 3) & 7)] + fw[10 + ((dc >> 6) & 7)] + ((dc >> 9) & 1);
      sh[u] = dc >> 10;
    }
    tj[u] = k < MK_BCC5_N ? ty[jj[u]] : 0;
    rj[u] = k < MK_BCC5_N + 2 ? rho[jj[u]] : 0.0;
  }
  // arguments and intervals of the (up to) four evaluations
  double x[4], t[4];
  int sp[4], ix[4];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int k = lane + 32 * u;
    if (k < MK_BCC5_N) {
      x[2 * u] = rj[u] + (sFd[sh[u] * K + tb] - sFd[sh[u] * K + ta]);
      x[2 * u + 1] = rj[u];
      sp[2 * u] = sp[2 * u + 1] = tj[u];
    } else {
      // the own-site terms: + F_tb(rho_i) (k = 58), - F_ta(rho_i) (k = 59)
      x[2 * u] = rj[u];
      x[2 * u + 1] = 0.0;
      sp[2 * u] = k == MK_BCC5_N ? tb : ta;
      sp[2 * u + 1] = 0;
    }
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) ix[e] = spline_locate(a.embed[sp[e]], x[e], t[e], a.err);
  Cubic c[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) c[e] = a.embed[sp[e]].c[ix[e]];
  double v = 0.0;
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int k = lane + 32 * u;
    const double f0 = fma(t[2 * u], fma(t[2 * u], fma(t[2 * u], c[2 * u].w, c[2 * u].z), c[2 * u].y), c[2 * u].x);
    const double f1 =
        fma(t[2 * u + 1], fma(t[2 * u + 1], fma(t[2 * u + 1], c[2 * u + 1].w, c[2 * u + 1].z), c[2 * u + 1].y),
            c[2 * u + 1].x);
    if (k < MK_BCC5_N) v += f0 - f1;
    else if (k == MK_BCC5_N) v += f0;
    else if (k == MK_BCC5_N + 1) v -= f0;
  }
  __syncwarp();  // fw is rewritten for the next open trial
  return v;
}


__global__ void k_multi_df(MultiArgs a, double* dF) {
  const int q = threadIdx.x;
  if (q >= a.K * a.K) return;
  const double r0 = a.rho[0];
  dF[q] = spline_val(a.embed[q % a.K], r0, a.err) - spline_val(a.embed[q / a.K], r0, a.err);
}

void launch_multi_df(const MultiArgs& a, double* dF, cudaStream_t st) { k_multi_df<<<1, 32, 0, st>>>(a, dF); }

__device__ __forceinline__ int multi_target(const MultiArgs& a, const MRepParams& p, long long step, int d, int ta) {
  if (a.K == 2) return 1 - ta;
  const uint4 w6 = philox4x32_10(make_uint4((uint32_t)step, (uint32_t)((uint64_t)step >> 32), (uint32_t)d, TAG_SPECIES),
                                 p.key);
  return (ta + 1 + (int)below64(w6.x, w6.y, (uint64_t)(a.K - 1))) % a.K;
}

// Surrogate descriptor of the site in cell (cx, cy, cz), basis b, species ti
// from the per-site shell counts: own[s] = B sites in shell s of the site;
// nb[s] = B sites other than the site itself in shell s of its 8 first-shell
// neighbours k, summed (the site is in shell 1 of each k).  The neighbours of
// a corner site (b = 0) are the body centres of the cells at offsets
// {-1, 0}^3, those of a body centre the corners at {0, 1}^3.  Eight 6-bit
// fields summed stay below 2^12: fields 0, 2, 4 and 1, 3 are summed in two
// words with 12 bits between fields.
__device__ __forceinline__ void multi_descriptor(const MultiArgs& a, int r, int cx, int cy, int cz, int b, int ti,
                                                 int (&own)[5], int (&nb)[5]) {
  const uint32_t* nc = a.nbc + (long long)r * a.rf_n;
  const long long row = (long long)a.qx * a.rf_q;
  const int lo = b ? 0 : -1;
  int xp[2], yv[2], zv[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int X = mk_wrap(cx + lo + q, a.nx), xq = X / a.qx;
    xp[q] = (X - xq * a.qx) * a.rf_q + xq;
    yv[q] = mk_wrap(cy + lo + q, a.ny);
    zv[q] = mk_wrap(cz + lo + q, a.nz);
  }
  const uint32_t w0 = nc[((long long)(b * a.nz + cz) * a.ny + cy) * row + (b ? xp[0] : xp[1])];
  const int nbb = 1 - b;
  uint32_t xs = 0u, ys = 0u;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const uint32_t w = nc[((long long)(nbb * a.nz + zv[q >> 2]) * a.ny + yv[(q >> 1) & 1]) * row + xp[q & 1]];
    xs += w & 0x3F03F03Fu;
    ys += (w >> 6) & 0x0003F03Fu;
  }
#pragma unroll
  for (int s = 0; s < 5; ++s) own[s] = (int)((w0 >> (6 * s)) & 63u);
  nb[0] = (int)(xs & 0xFFFu) - 8 * ti;
  nb[1] = (int)(ys & 0xFFFu);
  nb[2] = (int)((xs >> 12) & 0xFFFu);
  nb[3] = (int)(ys >> 12);
  nb[4] = (int)(xs >> 24);
}

// MODE 0: no re-embedding; 1: re-embedding, FP64 dE (any neighbour table);
// 2: re-embedding, five-shell table, FP32 screen (the dE sum of an accepted
// step is then taken by the commit launch, in FP64); 3: mode 2 with delayed
// acceptance (K = 2).  Modes 0 and 1 take their step from the replica's
// state and the last block of each replica takes the global decision; the
// screened modes take step *base + j and leave the decision to the commit
// launch, whose every block reads the step's complete sums.
template <int MODE>
__global__ void __launch_bounds__(MK_BLOCK, 4) k_multi_propose(MultiArgs a, int j) {
  constexpr bool REEMBED = MODE != 0;
  constexpr bool SCREEN = MODE >= 2;
  __shared__ double sV[MK_MAX_SH * MK_MAX * MK_MAX];
  __shared__ double sFd[MK_MAX_SH * MK_MAX];
  __shared__ double sDF[MK_MAX * MK_MAX];
  __shared__ long long sDq[5 * MK_MAX * MK_MAX * MK_MAX];
  __shared__ float sDfs[5 * MK_MAX * MK_MAX];
  // screened form: per-thread wrapped cell offsets and the block's
  // neighbour descriptors (unused otherwise)
  __shared__ int sw[SCREEN ? 30 * MK_BLOCK : 1];
  __shared__ int scode[SCREEN ? MK_BCC5_N : 1];
  __shared__ int s_fw[SCREEN ? MK_BLOCK / 32 : 1][15];
  // delayed acceptance: the block's stage-1 passes, queued for the exact
  // stage (site and cell; species, g, owner thread and trial), and the
  // owners' stage-2 decisions
  __shared__ int4 s_qa[MODE == 3 ? MK_BLOCK : 1];
  __shared__ int4 s_qb[MODE == 3 ? MK_BLOCK : 1];
  __shared__ int s_dec[MODE == 3 ? MK_BLOCK : 1];
  __shared__ int s_gw[MODE == 3 ? MK_BLOCK / MK_GROUP : 1][30];
  __shared__ uint64_t s_u2[MODE == 3 ? MK_BLOCK : 1];
  __shared__ int s_nq;
  __shared__ uint4 s_wc;
  __shared__ int s_col[4];
  __shared__ int s_red[MK_BLOCK / 32][MK_MAX + 1];
  __shared__ double s_de[MK_BLOCK / 32];
  __shared__ int s_s1[MK_BLOCK / 32];
  __shared__ bool s_last;
  // the global stage's inputs that no block of this step writes: the
  // replica's running state and beta kappa_p, n0 per solute
  __shared__ MRepState s_rs;
  __shared__ double s_bk[MK_MAX], s_n0[MK_MAX];
  const int K = a.K;
  for (int q = threadIdx.x; q < a.n_sh * K * K; q += MK_BLOCK) sV[q] = a.V[q];
  for (int q = threadIdx.x; q < a.n_sh * K; q += MK_BLOCK) sFd[q] = a.Fd[q];
  if (!REEMBED && threadIdx.x < K * K) sDF[threadIdx.x] = a.dF[threadIdx.x];
  if (a.bcc5)
    for (int q = threadIdx.x; q < 5 * K * K * K; q += MK_BLOCK) sDq[q] = a.Dq[q];
  if (SCREEN)
    for (int q = threadIdx.x; q < 5 * K * K; q += MK_BLOCK) {
      const int sh = q / (K * K), x = (q / K) % K, y = q % K;
      sDfs[q] = (float)(a.Fd[sh * K + y] - a.Fd[sh * K + x]);
    }
  const int r = blockIdx.y;
  const MRepParams& p = a.rp[r];
  const long long step = SCREEN ? *a.base + j : a.rs[r].step;
  if (threadIdx.x == 0) {
    // the step's colour (and global uniform), once per block
    const uint4 wc = philox4x32_10(make_uint4((uint32_t)step, (uint32_t)((uint64_t)step >> 32), 0xFFFFFFFFu, TAG_STEP),
                                   p.key);
    const int c = (int)below64(wc.x, wc.y, (uint64_t)a.n_colours);
    const int pc = c >> 1;
    s_wc = wc;
    s_col[0] = c;
    s_col[1] = pc % a.qx;
    s_col[2] = (pc / a.qx) % a.qy;
    s_col[3] = pc / (a.qx * a.qy);
    s_nq = 0;
    if (!SCREEN) s_rs = a.rs[r];
  }
  if (!SCREEN && threadIdx.x < MK_MAX) {
    s_bk[threadIdx.x] = p.beta * p.kappa_p[threadIdx.x];
    s_n0[threadIdx.x] = p.n0[threadIdx.x];
  }
  __syncthreads();
  const uint4 wc = s_wc;
  const int c = s_col[0];
  if constexpr (SCREEN) {
    if (threadIdx.x < MK_BCC5_N) {
      const int k = threadIdx.x;
      scode[k] = (c & 1) ? mk_bcc5_desc<1>(k) : mk_bcc5_desc<0>(k);
    }
    __syncthreads();
  }
  const int d = blockIdx.x * MK_BLOCK + threadIdx.x;
  int acc = 0, tie = 0, ta = 0, tb = 0, site = -1, dec = 0;
  double de = 0.0;
  long long pq = 0;
  uint64_t u53 = 0;
  // site of trial d (ascending index within the colour) and its draw: they
  // depend on no earlier launch
  const int b = c & 1;
  int cx = 0, cy = 0, cz = 0;
  if (d < a.D) {
    const int dq = mk_div(d, a.nxq, a.rcp_nxq);
    const int kx = d - dq * a.nxq;
    const int kz = mk_div(dq, a.nyq, a.rcp_nyq);
    const int ky = dq - kz * a.nyq;
    cx = s_col[1] + a.qx * kx;
    cy = s_col[2] + a.qy * ky;
    cz = s_col[3] + a.qz * kz;
    site = ((cz * a.ny + cy) * a.nx + cx) * 2 + b;
    const uint4 w = philox4x32_10(make_uint4((uint32_t)step, (uint32_t)((uint64_t)step >> 32), (uint32_t)d, TAG_TRIAL),
                                  p.key);
    u53 = top53(w.z, w.w);
    if constexpr (MODE == 3) {
      // delayed acceptance: the stage-2 uniform too, while the previous
      // launch drains
      const uint4 w2 = philox4x32_10(
          make_uint4((uint32_t)step, (uint32_t)((uint64_t)step >> 32), (uint32_t)d, TAG_STAGE2), p.key);
      s_u2[threadIdx.x] = top53(w2.x, w2.y);
    }
  }
  // screened form: launched after the previous step's commit with
  // programmatic dependent launch; the species, densities and this step's
  // accumulators are read after the wait (a no-op for an ordinary launch)
  if constexpr (SCREEN) pdl_wait();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int s1 = 0;
  if constexpr (MODE == 3) {
    // delayed acceptance (K = 2).  Stage 1 on the surrogate: every lane
    // takes part in the network (lanes without a trial feed zeros).
    uint32_t P[5] = {0u, 0u, 0u, 0u, 0u};
    if (d < a.D) {
      ta = a.types[(long long)r * a.N + site];
      tb = 1 - ta;
      int own[5], nb[5];
      multi_descriptor(a, r, cx, cy, cz, b, ta, own, nb);
      mlp_pairs(own, nb, P);
    }
    const float gnn = mlp_warp_eval_pair(a.mlp, P);
    if (d < a.D) {
      // u < min{1, exp[-beta (s g + s dmu0)]}
      const double sg = ta ? -1.0 : 1.0;
      s1 = metropolis(p.beta * fma(sg, p.dmu0[1], sg * (double)gnn), u53, &tie) ? 1 : 0;
    }
    // the block's stage-1 passes in one queue; warp w takes entries
    // 32 w .. 32 w + 31 for stage 2, so only ceil(passes / 32) warps
    // gather the exact dE's neighbourhood
    const unsigned pm = __ballot_sync(0xffffffffu, s1);
    if (pm) {
      int qb = 0;
      if (lane == 0) qb = atomicAdd(&s_nq, __popc(pm));
      qb = __shfl_sync(0xffffffffu, qb, 0);
      if (s1) {
        const int e = qb + __popc(pm & ((1u << lane) - 1u));
        s_qa[e] = make_int4(site, cx, cy, cz);
        s_qb[e] = make_int4(ta, __float_as_int(gnn), threadIdx.x, d);
      }
    }
    __syncthreads();
    const int nq = s_nq;
    int tie2 = 0;
    // stage 2: u2 < min{1, exp[-beta (dE - s g)]}, FP32-screened with the
    // bound of the plain rule's screen (FP64 by the warp where it cannot
    // decide).  Every group of MK_GROUP lanes takes one queued trial, so
    // the block's 128 threads screen 16 trials at a time.
    const int gl = threadIdx.x & (MK_GROUP - 1);
    for (int q0 = 0; q0 < nq; q0 += MK_BLOCK / MK_GROUP) {
      const int e = q0 + threadIdx.x / MK_GROUP;
      const bool has = e < nq;
      int4 qa = make_int4(0, 0, 0, 0), qo = make_int4(0, 0, 0, 0);
      if (has) {
        qa = s_qa[e];
        qo = s_qb[e];
      }
      long long qpq = 0;
      float err;
      bool in;
      const float e32 = multi_screen_group(a, sDq, sDfs, s_gw[threadIdx.x / MK_GROUP], scode, r, qa.x, qa.y, qa.z,
                                           qa.w, qo.x, 1 - qo.x, gl, has, &qpq, &err, &in);
      const bool lead = has && gl == 0;
      int dec2 = 0;
      uint64_t u2 = 0;
      if (lead) {
        u2 = s_u2[qo.z];
        const float g = __int_as_float(qo.y);
        // -s g (exact) plus the own-site offset of the FP32 tables: two
        // roundings, inside 2^-21 (|g| + |offset|)
        const float off = a.emb_off[qo.x * K + 1 - qo.x];
        const float cm = (qo.x ? g : -g) + off;
        const float x32 = p.beta32 * (e32 + cm);
        const float dx =
            p.beta32 * fmaf(4.76837158203125e-07f, fabsf(e32) + fabsf(g) + fabsf(off), err) * 1.0001f +
            fabsf(x32) * 4.76837158203125e-07f;
        dec2 = in ? screen32(x32, dx, u2) : -1;
      }
      unsigned open = __ballot_sync(0xffffffffu, lead && dec2 < 0);
      while (open) {
        const int src = __ffs(open) - 1;
        open &= open - 1u;
        const int si = __shfl_sync(0xffffffffu, qa.x, src);
        const int sa = __shfl_sync(0xffffffffu, qo.x, src);
        const double v = warp_sum(multi_emb_warp5(a, sFd, scode, s_fw[warp], r, si, sa, 1 - sa, lane));
        if (lane == src) {
          const double de64 = (double)qpq * a.qscale + v;
          if (!isfinite(de64)) atomicOr(a.err, ERRF_NONFINITE);
          const double sg = qo.x ? -1.0 : 1.0;
          dec2 = metropolis(p.beta * (de64 - sg * (double)__int_as_float(qo.y)), u2, &tie2) ? 1 : 0;
        }
      }
      if (lead) s_dec[qo.z] = dec2;
      __syncwarp();  // the group's scratch is rewritten by the next round
    }
    __syncthreads();
    acc = s1 ? s_dec[threadIdx.x] : 0;
    tie += tie2;
  } else if (d < a.D) {
    ta = a.types[(long long)r * a.N + site];
    tb = multi_target(a, p, step, d, ta);
    if constexpr (SCREEN) {
      float err;
      bool in;
      const float e32 = multi_screen_bcc5(a, sDq, sDfs, sw, scode, r, site, cx, cy, cz, ta, tb, &pq, &err, &in);
      const float cm = p.cmu32[ta * K + tb];
      const float x32 = p.beta32 * (e32 + cm);
      const float dx = p.beta32 * fmaf(4.76837158203125e-07f, fabsf(e32) + fabsf(cm), err) * 1.0001f +
                       fabsf(x32) * 4.76837158203125e-07f;
      dec = in ? screen32(x32, dx, u53) : -1;
      acc = dec > 0 ? 1 : 0;
    } else {
      if (a.bcc5)
        de = b ? multi_de_bcc5<1, REEMBED>(a, sDq, sFd, sDF, r, site, cx, cy, cz, ta, tb)
               : multi_de_bcc5<0, REEMBED>(a, sDq, sFd, sDF, r, site, cx, cy, cz, ta, tb);
      else
        de = multi_de<REEMBED>(a, sV, sFd, r, site, ta, tb);
      if (!isfinite(de)) atomicOr(a.err, ERRF_NONFINITE);
      acc = metropolis(p.beta * (de + (p.dmu0[tb] - p.dmu0[ta])), u53, &tie) ? 1 : 0;
    }
  }
  if constexpr (MODE == 2) {
    // trials the screen left open: FP64 dE by the whole warp, one at a time
    unsigned open = __ballot_sync(0xffffffffu, dec < 0);
    while (open) {
      const int src = __ffs(open) - 1;
      open &= open - 1u;
      const int si = __shfl_sync(0xffffffffu, site, src);
      const int sa = __shfl_sync(0xffffffffu, ta, src), sb = __shfl_sync(0xffffffffu, tb, src);
      const double v = warp_sum(multi_emb_warp5(a, sFd, scode, s_fw[warp], r, si, sa, sb, lane));
      if (lane == src) {
        const double de64 = (double)pq * a.qscale + v;
        if (!isfinite(de64)) atomicOr(a.err, ERRF_NONFINITE);
        acc = metropolis(p.beta * (de64 + (p.dmu0[tb] - p.dmu0[ta])), u53, &tie) ? 1 : 0;
      }
    }
  }
  MStepAcc* A = a.acc + 2 * r + (int)(step & 1);
  // compaction of the local accepts: one reservation per warp
  const unsigned m = __ballot_sync(0xffffffffu, acc);
  if (m) {
    int base = 0;
    if (lane == 0) base = atomicAdd(&A->nacc, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (acc) a.pend[(long long)r * a.D + base + __popc(m & ((1u << lane) - 1u))] = make_int2(site, tb | (ta << 8));
  }
  // per-solute dn, ties and the dE sum: warp, then block, then one atomic each
#pragma unroll
  for (int al = 1; al < MK_MAX; ++al) {
    const int v = acc ? (int)(tb == al) - (int)(ta == al) : 0;
    const int sv = __reduce_add_sync(0xffffffffu, v);
    if (lane == 0) s_red[warp][al] = sv;
  }
  const int st = __reduce_add_sync(0xffffffffu, tie);
  const int ss1 = MODE == 3 ? __reduce_add_sync(0xffffffffu, s1) : 0;
  double sd = (!SCREEN && acc) ? de : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, o);
  if (lane == 0) {
    s_red[warp][0] = st;
    s_de[warp] = sd;
    s_s1[warp] = ss1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int tsum = 0, s1sum = 0;
    double dsum = 0.0;
    for (int w = 0; w < MK_BLOCK / 32; ++w) {
      tsum += s_red[w][0];
      dsum += s_de[w];
      s1sum += s_s1[w];
    }
    if (s1sum) atomicAdd(&A->s1, s1sum);
    for (int al = 1; al < K; ++al) {
      int v = 0;
      for (int w = 0; w < MK_BLOCK / 32; ++w) v += s_red[w][al];
      if (v) atomicAdd(&A->dn[al], v);
    }
    if (tsum) atomicAdd(&A->ties, tsum);
    if (dsum != 0.0) atomicAdd(&A->sum_de, dsum);
    if (!SCREEN) {
      __threadfence();
      s_last = atomicAdd(&A->done, 1u) == gridDim.x - 1;
    }
  }
  // screened forms: the commit launch takes the global decision
  if constexpr (SCREEN) return;
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  // global stage (last block of the replica): every block's sums are
  // visible; they are loaded in one round
  __threadfence();
  const int nacc = __ldcg(&A->nacc);
  const int ties = __ldcg(&A->ties);
  const int s1v = MODE == 3 ? __ldcg(&A->s1) : 0;
  const double sde = __ldcg(&A->sum_de);
  int dn[MK_MAX];
#pragma unroll
  for (int al = 1; al < MK_MAX; ++al) dn[al] = al < K ? __ldcg(&A->dn[al]) : 0;
  MRepState s = s_rs;
  s.trials += a.D;
  s.local_acc += nacc;
  s.near_ties += ties;
  s.s1_acc += s1v;
  int accept = 0;
  if (nacc > 0) {
    s.global_trials++;
    double Y = 0.0;
#pragma unroll
    for (int al = 1; al < MK_MAX; ++al)
      if (al < K) Y += s_bk[al] * (double)dn[al] * ((double)dn[al] + 2.0 * ((double)s.cnt[al] - s_n0[al]));
    int gtie = 0;
    accept = metropolis(Y, top53(wc.z, wc.w), &gtie) ? 1 : 0;
    s.near_ties += gtie;
    if (accept) {
      s.global_acc++;
      s.flips += nacc;
      long long d0 = 0;
#pragma unroll
      for (int al = 1; al < MK_MAX; ++al)
        if (al < K) {
          s.cnt[al] += dn[al];
          d0 += dn[al];
        }
      s.cnt[0] -= d0;
      s.energy += sde;
    }
  }
  A->accept = accept;
  A->done = 0u;
  s.steps++;
#pragma unroll
  for (int al = 0; al < MK_MAX; ++al)
    if (al < K) {
      const double cc = (double)s.cnt[al] * a.inv_n;
      s.sum_c[al] += cc;
      s.sum_c2[al] += cc * cc;
    }
  s.step++;
  a.rs[r] = s;
}

// apply an accepted step: species, and the density change of the neighbours
// (pend entries: site, new species | old species << 8)
template <int MODE>
__global__ void __launch_bounds__(MK_BLOCK) k_multi_commit(MultiArgs a) {
  const int r = blockIdx.y;
  const long long step = a.rs[r].step - 1;  // the step the propose launch decided
  const MStepAcc* A = a.acc + 2 * r + (int)(step & 1);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // the other buffer takes the next step's sums
    MStepAcc* B = a.acc + 2 * r + (int)((step + 1) & 1);
    for (int al = 0; al < MK_MAX; ++al) B->dn[al] = 0;
    B->nacc = 0;
    B->ties = 0;
    B->accept = 0;
    B->s1 = 0;
    B->sum_de = 0.0;
  }
  if (!A->accept) return;
  const int nacc = A->nacc;
  uint8_t* ty = a.types + (long long)r * a.N;
  double* rho = a.rho + (long long)r * a.N;
  for (int q = blockIdx.x * MK_BLOCK + threadIdx.x; q < nacc; q += gridDim.x * MK_BLOCK) {
    const int2 e = a.pend[(long long)r * a.D + q];
    const int tb = e.y & 255, ta = e.y >> 8;
    ty[e.x] = (uint8_t)tb;
    if constexpr (MODE == 1) {
      const int3 p = multi_half(a, e.x);
      for (int k = 0; k < a.n_off; ++k) {
        const int4 h = a.off[k];
        rho[multi_nbr_at(a, p, h)] += a.Fd[h.w * a.K + tb] - a.Fd[h.w * a.K + ta];
      }
    }
  }
}

// Screened form: one thread per (accept, neighbour) and one per accepted
// site over all replicas that accepted their step, on a fixed grid: the
// density change in FP64 with its float copy and the FP32 embedding value
// there, and the new species with its embedding value.  Accepts of one step
// are more than 2 r_c apart: no two threads touch a common site, and no
// neighbour's species changes.  Every block sums the replicas' item counts
// (at most MK_SCREEN_MAX_R replicas; the host selects this form only while
// R D (MK_BCC5_N + 1) < 2^31, so the int item index cannot overflow).
__global__ void __launch_bounds__(MK_BLOCK) k_multi_commit_screen(MultiArgs a, int jl) {
  // the next step's propose may start its draws now; it reads what this
  // launch writes only after griddepcontrol.wait
  pdl_trigger();
  __shared__ int s_pre[MK_SCREEN_MAX_R + 1];
  __shared__ int4 s_off[MK_BCC5_N];
  __shared__ double s_df[5 * MK_MAX * MK_MAX];
  const int K = a.K;
  constexpr int NI = MK_BCC5_N + 1;
  const long long step = *a.base + jl;  // the step the propose launch proposed
  // the global stage of every replica (Eq. trans_vcsgc_par2 per solute),
  // taken in every block from the step's complete sums: the same FP64
  // arithmetic everywhere, so the same decision.  Block 0 folds the step
  // into the replica's state and readies the next step's accumulator.
  for (int r = threadIdx.x; r < a.R; r += MK_BLOCK) {
    const MStepAcc* A = a.acc + 2 * r + (int)(step & 1);
    const MRepParams& p = a.rp[r];
    const int nacc = __ldcg(&A->nacc);
    int dn[MK_MAX];
    long long c0[MK_MAX];
#pragma unroll
    for (int al = 0; al < MK_MAX; ++al) {
      dn[al] = al > 0 && al < K ? __ldcg(&A->dn[al]) : 0;
      c0[al] = al < K ? __ldcg(&A->cnt[al]) : 0;
    }
    int accept = 0, gtie = 0;
    if (nacc > 0) {
      double Y = 0.0;
#pragma unroll
      for (int al = 1; al < MK_MAX; ++al)
        if (al < K)
          Y += p.beta * p.kappa_p[al] * (double)dn[al] * ((double)dn[al] + 2.0 * ((double)c0[al] - p.n0[al]));
      const uint4 wc = philox4x32_10(
          make_uint4((uint32_t)step, (uint32_t)((uint64_t)step >> 32), 0xFFFFFFFFu, TAG_STEP), p.key);
      accept = metropolis(Y, top53(wc.z, wc.w), &gtie) ? 1 : 0;
    }
    s_pre[r + 1] = accept ? nacc * NI : 0;
    if (blockIdx.x == 0) {
      MRepState s = a.rs[r];
      s.trials += a.D;
      s.local_acc += nacc;
      s.near_ties += __ldcg(&A->ties) + gtie;
      s.s1_acc += __ldcg(&A->s1);
      if (nacc > 0) {
        s.global_trials++;
        if (accept) {
          s.global_acc++;
          s.flips += nacc;
          long long d0 = 0;
#pragma unroll
          for (int al = 1; al < MK_MAX; ++al)
            if (al < K) {
              s.cnt[al] += dn[al];
              d0 += dn[al];
            }
          s.cnt[0] -= d0;
        }
      }
      s.steps++;
#pragma unroll
      for (int al = 0; al < MK_MAX; ++al)
        if (al < K) {
          const double cc = (double)s.cnt[al] * a.inv_n;
          s.sum_c[al] += cc;
          s.sum_c2[al] += cc * cc;
        }
      s.step = step + 1;
      a.rs[r] = s;
      MStepAcc* B = a.acc + 2 * r + (int)((step + 1) & 1);
#pragma unroll
      for (int al = 0; al < MK_MAX; ++al) {
        B->dn[al] = 0;
        B->cnt[al] = s.cnt[al];
      }
      B->nacc = 0;
      B->ties = 0;
      B->done = 0u;
      B->accept = 0;
      B->s1 = 0;
      B->sum_de = 0.0;
    }
  }
  for (int q = threadIdx.x; q < MK_BCC5_N; q += MK_BLOCK) s_off[q] = a.off[q];
  for (int q = threadIdx.x; q < 5 * K * K; q += MK_BLOCK) {
    const int sh = q / (K * K), x = (q / K) % K, y = q % K;
    s_df[q] = a.Fd[sh * K + y] - a.Fd[sh * K + x];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s_pre[0] = 0;
    for (int r = 0; r < a.R; ++r) s_pre[r + 1] += s_pre[r];
  }
  __syncthreads();
  const int total = s_pre[a.R];
  int r = 0;
  for (int it = blockIdx.x * MK_BLOCK + threadIdx.x; it < total; it += gridDim.x * MK_BLOCK) {
    while (s_pre[r + 1] <= it) ++r;
    const int loc = it - s_pre[r];
    const int q = loc / NI, k = loc - q * NI;
    const int2 e = a.pend[(long long)r * a.D + q];
    const int tb = e.y & 255, ta = e.y >> 8;
    uint8_t* ty = a.types + (long long)r * a.N;
    float2* rf = a.rf + (long long)r * a.rf_n;
    const int3 ph = multi_half(a, e.x);
    if (k < MK_BCC5_N) {
      const int4 h = s_off[k];
      int X, Y, Z, bb;
      multi_nbr_cell(a, ph, h, X, Y, Z, bb);
      const int j = ((Z * a.ny + Y) * a.nx + X) * 2 + bb;
      double* rho = a.rho + (long long)r * a.N;
      const double nr = rho[j] + s_df[(h.w * K + ta) * K + tb];
      rho[j] = nr;
      const float r32 = (float)nr;
      const long long q = multi_rfi(a, X, Y, Z, bb);
      rf[q] = make_float2(r32, emb32_val(a, ty[j], r32));
      // delayed acceptance (K = 2): the flipped site is in shell h.w of j
      if (a.da) a.nbc[(long long)r * a.rf_n + q] += (uint32_t)(tb - ta) << (6 * h.w);
    } else {
      ty[e.x] = (uint8_t)tb;
      const int b = e.x & 1;
      const long long q = multi_rfi(a, (ph.x - b) >> 1, (ph.y - b) >> 1, (ph.z - b) >> 1, b);
      rf[q].y = emb32_val(a, tb, rf[q].x);
    }
  }
}

void launch_multi_step(const MultiArgs& a, int j, cudaStream_t st, bool after_step) {
  const int nb = (a.D + MK_BLOCK - 1) / MK_BLOCK;
  const dim3 grid((unsigned)nb, (unsigned)a.R);
  // the accepts of a step are a small share of its trials: a few blocks per
  // replica stride over them
  const dim3 cgrid((unsigned)(nb < 4 ? nb : 4), (unsigned)a.R);
  if (a.screen) {
    // one thread per (accept, neighbour) over all replicas: a fixed grid of
    // four blocks per SM
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(MK_BLOCK);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = after_step ? 1 : 0;
    if (a.da)
      cudaLaunchKernelEx(&cfg, k_multi_propose<3>, a, j);
    else
      cudaLaunchKernelEx(&cfg, k_multi_propose<2>, a, j);
    k_multi_commit_screen<<<4 * a.n_sm, MK_BLOCK, 0, st>>>(a, j);
  } else if (a.reembed) {
    k_multi_propose<1><<<grid, MK_BLOCK, 0, st>>>(a, 0);
    k_multi_commit<1><<<cgrid, MK_BLOCK, 0, st>>>(a);
  } else {
    k_multi_propose<0><<<grid, MK_BLOCK, 0, st>>>(a, 0);
    k_multi_commit<0><<<cgrid, MK_BLOCK, 0, st>>>(a);
  }
}

// ------------------------------------------------------------ fused form
// One launch per colour step k (no re-embedding, five-shell table):
//  1. every block takes the global decision of step k - 1 from that step's
//     sums (the same FP64 arithmetic in every block, so the same result);
//  2. each thread commits its pending flip of step k - 1 (slot d): the new
//     species if the step was accepted, else the old one;
//  3. block 0 of the replica folds step k - 1 into the running state;
//  4. each thread proposes trial d of step k on the effective species: a
//     neighbour whose byte still carries a pending flip of step k - 1 counts
//     with its new species when that step was accepted, so the commits of
//     other blocks need not have landed;
//  5. an accepted trial marks its site pending (high nibble) and its slot.
// Concurrent readers see either the byte before its commit (species and
// pending) or after (the committed species): both give the same effective
// species.  Same-colour sites are more than 2 r_c apart, so no trial reads
// another trial of its own step.
// neighbour bytes of the site in cell (cx, cy, cz), basis B: all 58 loads
// issued at once
template <int B>
__device__ __forceinline__ void multi_bytes(const MultiArgs& a, const uint8_t* ty, int cx, int cy, int cz,
                                            unsigned* by) {
  int xo[5], yo[5], zo[5];
#pragma unroll
  for (int dd = -2; dd <= 2; ++dd) {
    xo[dd + 2] = 2 * mk_wrap(cx + dd, a.nx);
    yo[dd + 2] = 2 * a.nx * mk_wrap(cy + dd, a.ny);
    zo[dd + 2] = 2 * a.nx * a.ny * mk_wrap(cz + dd, a.nz);
  }
#pragma unroll
  for (int k = 0; k < MK_BCC5_N; ++k) {
    const int code = mk_bcc5_code(k);
    const int hx = (code & 15) - 4, hy = ((code >> 4) & 15) - 4, hz = ((code >> 8) & 15) - 4;
    const int bb = B ^ (hx & 1);
    by[k] = __ldcg(ty + zo[((B + hz - bb) >> 1) + 2] + yo[((B + hy - bb) >> 1) + 2] + xo[((B + hx - bb) >> 1) + 2] + bb);
  }
}

// pair part of dE in fixed point from the neighbour bytes and the effective
// species (gmask = 0xF0 when the previous step was accepted: a pending
// nibble then counts)
__device__ __forceinline__ long long multi_pq_bytes(const MultiArgs& a, const long long* sDq, const unsigned* by,
                                                    unsigned gmask, int ta, int tb) {
  const int K = a.K;
  unsigned cnt[5] = {0u, 0u, 0u, 0u, 0u};
#pragma unroll
  for (int k = 0; k < MK_BCC5_N; ++k) {
    const unsigned v = by[k];
    const unsigned te = (v & gmask) ? (v >> 4) - 1u : (v & 15u);
    cnt[mk_bcc5_code(k) >> 12] += 1u << (8 * te);
  }
  long long pq = 0;
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const long long* D = sDq + ((s * K + ta) * K + tb) * K;
    for (int be = 0; be < K; ++be) pq += (long long)((cnt[s] >> (8 * be)) & 255u) * D[be];
  }
  return pq;
}

// Launches of a chain after the first use programmatic dependent launch:
// before griddepcontrol.wait a step reads only what no step writes (the
// tables, the parameters, the step base, which only the advance kernel
// changes and the first launch after it is ordinary) and draws its random
// numbers; what the previous step wrote is read after the wait.
template <bool PROPOSE>
__global__ void __launch_bounds__(MK_BLOCK) k_multi_fused(MultiArgs a, int j) {
  pdl_trigger();
  __shared__ long long sDq[5 * MK_MAX * MK_MAX * MK_MAX];
  __shared__ double sDF[MK_MAX * MK_MAX];
  __shared__ int s_G, s_tie;
  __shared__ int s_red[MK_BLOCK / 32][MK_MAX + 1];
  __shared__ double s_de[MK_BLOCK / 32];
  __shared__ int s_acc[MK_BLOCK / 32];
  const int K = a.K;
  const int r = blockIdx.y;
  const MRepParams& p = a.rp[r];
  const long long k = *a.base + j, kp = k - 1;
  const int d = blockIdx.x * MK_BLOCK + threadIdx.x;
  if (PROPOSE) {
    for (int q = threadIdx.x; q < 5 * K * K * K; q += MK_BLOCK) sDq[q] = a.Dq[q];
    if (threadIdx.x < K * K) sDF[threadIdx.x] = a.dF[threadIdx.x];
  }
  // draws and the site of trial d of step k; the global uniform of step k-1
  uint64_t ug = 0;
  if (threadIdx.x == 0 && kp >= 0) {
    const uint4 wp = philox4x32_10(make_uint4((uint32_t)kp, (uint32_t)((uint64_t)kp >> 32), 0xFFFFFFFFu, TAG_STEP),
                                   p.key);
    ug = top53(wp.z, wp.w);
  }
  int site = -1, b = 0, cx = 0, cy = 0, cz = 0, toff = 0;
  uint64_t u53 = 0;
  if (PROPOSE && d < a.D) {
    const uint4 wc = philox4x32_10(make_uint4((uint32_t)k, (uint32_t)((uint64_t)k >> 32), 0xFFFFFFFFu, TAG_STEP),
                                   p.key);
    const int c = (int)below64(wc.x, wc.y, (uint64_t)a.n_colours);
    const int pc = c >> 1;
    b = c & 1;
    const int dq = mk_div(d, a.nxq, a.rcp_nxq);
    const int kx = d - dq * a.nxq;
    const int kz = mk_div(dq, a.nyq, a.rcp_nyq);
    const int ky = dq - kz * a.nyq;
    cx = pc % a.qx + a.qx * kx;
    cy = (pc / a.qx) % a.qy + a.qy * ky;
    cz = pc / (a.qx * a.qy) + a.qz * kz;
    site = ((cz * a.ny + cy) * a.nx + cx) * 2 + b;
    const uint4 w = philox4x32_10(make_uint4((uint32_t)k, (uint32_t)((uint64_t)k >> 32), (uint32_t)d, TAG_TRIAL),
                                  p.key);
    u53 = top53(w.z, w.w);
    if (K > 2) {
      const uint4 w6 = philox4x32_10(
          make_uint4((uint32_t)k, (uint32_t)((uint64_t)k >> 32), (uint32_t)d, TAG_SPECIES), p.key);
      toff = (int)below64(w6.x, w6.y, (uint64_t)(K - 1));
    }
  }
  pdl_wait();

  // loads of what the previous steps wrote, all before the block barrier
  uint8_t* ty = a.types + (long long)r * a.N;
  int* slot = a.slot + (long long)r * a.D + d;
  int ps = -1;
  unsigned vps = 0u, vown = 0u;
  unsigned by[MK_BCC5_N];
  if (d < a.D) {
    ps = __ldcg(slot);
    if (ps >= 0) vps = __ldcg(ty + ps);
  }
  if (site >= 0) {
    vown = __ldcg(ty + site);
    if (b) multi_bytes<1>(a, ty, cx, cy, cz, by);
    else multi_bytes<0>(a, ty, cx, cy, cz, by);
  }
  if (threadIdx.x == 0) {
    // global decision of step k-1 (every block, the same FP64 arithmetic)
    int G = 0, tie = 0;
    if (kp >= 0) {
      const MStepAcc* A = a.acc + 3 * r + (int)(kp % 3);
      if (__ldcg(&A->nacc) > 0) {
        const long long* n0 = a.nstart + (2 * r + (int)(kp & 1)) * MK_MAX;
        double Y = 0.0;
        for (int al = 1; al < K; ++al) {
          const double dn = (double)__ldcg(&A->dn[al]);
          Y += p.beta * p.kappa_p[al] * dn * (dn + 2.0 * ((double)__ldcg(n0 + al) - p.n0[al]));
        }
        G = metropolis(Y, ug, &tie) ? 1 : 0;
      }
    }
    s_G = G;
    s_tie = tie;
  }
  __syncthreads();
  const int G = s_G;
  const unsigned gmask = G ? 0xF0u : 0u;
  // commit this thread's pending flip of step k-1
  if (ps >= 0) ty[ps] = (uint8_t)((vps & gmask) ? (vps >> 4) - 1u : (vps & 15u));
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    MRepState S = a.rs[r];
    if (kp >= 0 && S.fin_step < kp) {
      const MStepAcc* A = a.acc + 3 * r + (int)(kp % 3);
      const int nacc = __ldcg(&A->nacc);
      const long long* n0 = a.nstart + (2 * r + (int)(kp & 1)) * MK_MAX;
      long long cnt[MK_MAX];
      for (int al = 0; al < MK_MAX; ++al) cnt[al] = __ldcg(n0 + al);
      S.trials += a.D;
      S.local_acc += nacc;
      S.near_ties += __ldcg(&A->ties) + s_tie;
      if (nacc > 0) {
        S.global_trials++;
        if (G) {
          S.global_acc++;
          S.flips += nacc;
          long long d0 = 0;
          for (int al = 1; al < K; ++al) {
            const int dn = __ldcg(&A->dn[al]);
            cnt[al] += dn;
            d0 += dn;
          }
          cnt[0] -= d0;
          S.energy += __ldcg(&A->sum_de);
        }
      }
      long long* n1 = a.nstart + (2 * r + (int)(k & 1)) * MK_MAX;
      for (int al = 0; al < K; ++al) {
        S.cnt[al] = cnt[al];
        n1[al] = cnt[al];
        const double cc = (double)cnt[al] * a.inv_n;
        S.sum_c[al] += cc;
        S.sum_c2[al] += cc * cc;
      }
      S.steps++;
      S.step = k;
      S.fin_step = kp;
      a.rs[r] = S;
    }
    if (PROPOSE) {
      MStepAcc* Bn = a.acc + 3 * r + (int)((k + 1) % 3);
      for (int al = 0; al < MK_MAX; ++al) Bn->dn[al] = 0;
      Bn->nacc = 0;
      Bn->ties = 0;
      Bn->sum_de = 0.0;
    }
  }
  if (!PROPOSE) {
    if (ps >= 0) *slot = -1;
    return;
  }
  int acc = 0, tie = 0, ta = 0, tb = 0;
  double de = 0.0;
  if (site >= 0) {
    // the site's own byte may carry this thread's pending flip of step k-1
    ta = (int)((vown & gmask) ? (vown >> 4) - 1u : (vown & 15u));
    tb = K == 2 ? 1 - ta : (ta + 1 + toff) % K;
    const long long pq = multi_pq_bytes(a, sDq, by, gmask, ta, tb);
    // FP32 screen of u < min{1, exp(-X)}, X = beta (dE + dmu0_b - dmu0_a):
    // the pair part and the constant rounded to float, |x32 - X| bounded by
    // their size times 2^-21; FP64 only when the screen cannot decide
    const float e32 = (float)pq * (float)a.qscale, c32 = p.c32[ta * K + tb];
    const float x32 = p.beta32 * (e32 + c32);
    const float dx = (p.beta32 * (fabsf(e32) + fabsf(c32)) + fabsf(x32)) * 4.76837158203125e-07f;
    const int dec = screen32(x32, dx, u53);
    if (dec >= 0) {
      acc = dec;
    } else {
      const double d64 = (double)pq * a.qscale + sDF[ta * K + tb];
      acc = metropolis(p.beta * (d64 + (p.dmu0[tb] - p.dmu0[ta])), u53, &tie) ? 1 : 0;
    }
    if (acc) {
      de = (double)pq * a.qscale + sDF[ta * K + tb];
      if (!isfinite(de)) atomicOr(a.err, ERRF_NONFINITE);
    }
    if (acc) {
      ty[site] = (uint8_t)(ta | ((tb + 1) << 4));
      *slot = site;
    } else if (ps >= 0) {
      *slot = -1;
    }
  } else if (ps >= 0) {
    *slot = -1;
  }
  // per-solute dn, accepts, ties and the dE sum: warp, block, one atomic each
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int al = 1; al < MK_MAX; ++al) {
    const int sv = __reduce_add_sync(0xffffffffu, acc ? (int)(tb == al) - (int)(ta == al) : 0);
    if (lane == 0) s_red[warp][al] = sv;
  }
  const int sa = __reduce_add_sync(0xffffffffu, acc);
  const int st = __reduce_add_sync(0xffffffffu, tie);
  double sd = acc ? de : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, o);
  if (lane == 0) {
    s_red[warp][0] = st;
    s_acc[warp] = sa;
    s_de[warp] = sd;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int na = 0, nt = 0;
    double dsum = 0.0;
    for (int w2 = 0; w2 < MK_BLOCK / 32; ++w2) {
      na += s_acc[w2];
      nt += s_red[w2][0];
      dsum += s_de[w2];
    }
    MStepAcc* A = a.acc + 3 * r + (int)(k % 3);
    if (na) {
      atomicAdd(&A->nacc, na);
      for (int al = 1; al < K; ++al) {
        int v = 0;
        for (int w2 = 0; w2 < MK_BLOCK / 32; ++w2) v += s_red[w2][al];
        if (v) atomicAdd(&A->dn[al], v);
      }
      atomicAdd(&A->sum_de, dsum);
    }
    if (nt) atomicAdd(&A->ties, nt);
  }
}

__global__ void k_multi_advance(long long* base, int n) { *base += n; }

void launch_multi_fused(const MultiArgs& a, int j, bool propose, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((a.D + MK_BLOCK - 1) / MK_BLOCK), (unsigned)a.R);
  cfg.blockDim = dim3(MK_BLOCK);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = (propose && j > 0) ? 1 : 0;  // the first launch of a chain is ordinary
  if (propose) cudaLaunchKernelEx(&cfg, k_multi_fused<true>, a, j);
  else cudaLaunchKernelEx(&cfg, k_multi_fused<false>, a, j);
}

void launch_multi_advance(long long* base, int n, cudaStream_t st) { k_multi_advance<<<1, 1, 0, st>>>(base, n); }

__global__ void k_multi_delta_e(MultiArgs a, int r, const long long* sites, const uint8_t* to, int n, double* out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int i = (int)sites[q];
  const int ta = a.types[(long long)r * a.N + i], tb = to[q];
  out[q] = ta == tb ? 0.0
                    : (a.reembed ? multi_de<true>(a, a.V, a.Fd, r, i, ta, tb) : multi_de<false>(a, a.V, a.Fd, r, i, ta, tb));
}

void launch_multi_delta_e(const MultiArgs& a, int r, const long long* sites, const uint8_t* to, int n, double* out,
                          cudaStream_t st) {
  if (n <= 0) return;
  k_multi_delta_e<<<(n + 127) / 128, 128, 0, st>>>(a, r, sites, to, n, out);
}

// Delayed acceptance (K = 2): per-site B counts in the five shells from the
// species of every replica (shell s at bit 6 s of nbc, laid out like rf)
__global__ void k_multi_nbc(MultiArgs a) {
  const int r = blockIdx.y;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  const uint8_t* ty = a.types + (long long)r * a.N;
  uint32_t w = 0u;
  for (int k = 0; k < a.n_off; ++k) {
    const int4 h = a.off[k];
    w += (uint32_t)(ty[multi_nbr(a, (int)i, h)] == 1) << (6 * h.w);
  }
  const int3 p = multi_half(a, (int)i);
  const int b = (int)(i & 1);
  a.nbc[(long long)r * a.rf_n + multi_rfi(a, (p.x - b) >> 1, (p.y - b) >> 1, (p.z - b) >> 1, b)] = w;
}

void launch_multi_nbc(const MultiArgs& a, cudaStream_t st) {
  const dim3 grid((unsigned)((a.N + 255) / 256), (unsigned)a.R);
  k_multi_nbc<<<grid, 256, 0, st>>>(a);
}

// Surrogate descriptors X[r N + i][10] (raw counts from nbc) and targets
// Y[r N + i] = E(i = B) - E(i = A) (FP64 dE with re-embedding, rounded to
// float) of every site of every replica
__global__ void k_multi_features(MultiArgs a, float* X, float* Y) {
  const int r = blockIdx.y;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  const int ti = a.types[(long long)r * a.N + i];
  const int3 p = multi_half(a, (int)i);
  const int b = (int)(i & 1);
  int own[5], nb[5];
  multi_descriptor(a, r, (p.x - b) >> 1, (p.y - b) >> 1, (p.z - b) >> 1, b, ti, own, nb);
  const long long row = (long long)r * a.N + i;
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    X[row * 10 + s] = (float)own[s];
    X[row * 10 + 5 + s] = (float)nb[s];
  }
  const double de = multi_de<true>(a, a.V, a.Fd, r, (int)i, ti, 1 - ti);
  if (!isfinite(de)) atomicOr(a.err, ERRF_NONFINITE);
  Y[row] = (float)(ti == 0 ? de : -de);
}

void launch_multi_features(const MultiArgs& a, float* X, float* Y, cudaStream_t st) {
  const dim3 grid((unsigned)((a.N + 127) / 128), (unsigned)a.R);
  k_multi_features<<<grid, 128, 0, st>>>(a, X, Y);
}

}  // namespace vcsgc
