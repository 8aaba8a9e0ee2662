// kernels_mc.cu -- the colour step of the parallel VC-SGC method
// (Sec. III B 2 of Sadigh et al.): site pick, energy difference, local
// Metropolis stage, reduction of the concentration change, global stage and
// commit.  One colour step is two launches:
//   k_propose: every domain of the drawn colour picks a site, evaluates
//              dE_i and the local test (Eq. trans_vcsgc_par1); accepted
//              sites are compacted into a list and dn = sum s_i is reduced
//              (warp shuffles, one atomic per block: the paper's allgather);
//   k_commit:  every block derives the same global decision
//              (Eq. trans_vcsgc_par2, exponent -beta kappa_p dn (dn + 2(n-n0)))
//              and, if accepted, flips its share of the list and scatters the
//              density change; the last block to finish advances the
//              replica's counters.
// On the rigid lattice with species-dependent densities the local test is
// FP32-screened (delta_e_screen) and the commit runs one thread per
// (accept, neighbour).
#include "common.cuh"
#include "kernels.h"

namespace vcsgc {


// Energy change of flipping site i of replica r, t -> t' = 1 - t:
//   pair:     sum_k [phi_{t' t_k} - phi_{t t_k}](r_ik)
//   own:      F_{t'}(rho_i) - F_t(rho_i)
//   re-embed: sum_k F_{t_k}(rho_k + drho_k) - F_{t_k}(rho_k),
//             drho_k = f_{t'}(r_ik) - f_t(r_ik)
// SHELL: rigid lattice, slots grouped by shell so the pair sum is the
// per-shell B count times a tabulated difference (exact in arithmetic, no
// per-neighbour interpolation).  !SHELL: distances from positions.
template <bool SHELL, bool REEMBED>
__device__ double delta_e(const McArgs& a, int r, int i, unsigned* err) {
  const uint8_t* ty = a.types + (long long)r * a.N;
  const int t = ty[i];
  const int* row = a.nbr + (long long)i * a.K;
  double de;
  if constexpr (SHELL) {
    const int S = a.n_shells;
    de = a.shell_tab[0];
    int k = 0;
    for (int s = 0; s < S; ++s) {
      int cnt = 0;
      const int end = a.shell_end[s];
      for (; k < end; ++k) cnt += ty[row[k]];
      de = fma((double)cnt, a.shell_tab[1 + s], de);
    }
    if (t) de = -de;
    if constexpr (!REEMBED) {
      const double dfi = a.dF[i];
      de += t ? -dfi : dfi;
    } else {
      const double* rho = a.rho + (a.rho_per_rep ? (long long)r * a.N : 0);
      const double ri = rho[i];
      de += spline_val(a.tab.sp[6 - t], ri, err) - spline_val(a.tab.sp[5 + t], ri, err);
      k = 0;
      for (int s = 0; s < S; ++s) {
        const double dfs = a.shell_tab[1 + S + s];
        const double drho = t ? -dfs : dfs;
        const int end = a.shell_end[s];
        for (; k < end; ++k) {
          const int j = row[k];
          const int tj = ty[j];
          const double rj = rho[j];
          de += spline_val(a.tab.sp[5 + tj], rj + drho, err) - spline_val(a.tab.sp[5 + tj], rj, err);
        }
      }
    }
  } else {
    const int tp = 1 - t;
    const int cnt = a.nbr_cnt[i];
    const double xi = a.x[i], yi = a.y[i], zi = a.z[i];
    const long long hb[3] = {half_bits(a.box[0]), half_bits(a.box[1]), half_bits(a.box[2])};
    const double* rho = a.rho + (a.rho_per_rep ? (long long)r * a.N : 0);
    double pair = 0.0, re = 0.0;
    for (int k = 0; k < cnt; ++k) {
      const int j = row[k];
      const double dx = mimg_w(a.x[j] - xi, a.box[0], hb[0]);
      const double dy = mimg_w(a.y[j] - yi, a.box[1], hb[1]);
      const double dz = mimg_w(a.z[j] - zi, a.box[2], hb[2]);
      const double rr = sqrt(dx * dx + dy * dy + dz * dz);
      if (rr >= a.rc) continue;
      const int tj = ty[j];
      double tt;
      const int jj = spline_locate(a.tab.sp[0], rr, tt, err);
      pair += spline_val_at(a.tab.sp[tp + tj], jj, tt) - spline_val_at(a.tab.sp[t + tj], jj, tt);
      if constexpr (REEMBED) {
        const double drho = spline_val_at(a.tab.sp[3 + tp], jj, tt) - spline_val_at(a.tab.sp[3 + t], jj, tt);
        const double rj = rho[j];
        re += spline_val(a.tab.sp[5 + tj], rj + drho, err) - spline_val(a.tab.sp[5 + tj], rj, err);
      }
    }
    double own;
    if constexpr (REEMBED) {
      const double ri = rho[i];
      own = spline_val(a.tab.sp[5 + tp], ri, err) - spline_val(a.tab.sp[5 + t], ri, err);
    } else {
      own = t ? -a.dF[i] : a.dF[i];
    }
    de = pair + own + re;
  }
  return de;
}

// The general (explicit-position) form of dE by one warp: lanes take
// neighbours k = lane, lane + 32, ...; partial sums meet in a shuffle tree.
// Every lane returns the total.  The neighbours come in chunks of 96, three
// per lane, whose list entries, then positions and species, then table
// cubics load together (each lane adds its neighbours in the order k, as a
// one-at-a-time loop would).
constexpr int MCW_SLOTS = 3;

template <bool REEMBED, bool MIXED>
__device__ double delta_e_warp(const McArgs& a, int r, int i, int lane, unsigned* err) {
  const uint8_t* ty = a.types + (long long)r * a.N;
  const int t = ty[i];
  const int tp = 1 - t;
  const int* row = a.nbr + (long long)i * a.K;
  const int cnt = a.nbr_cnt[i];
  // FP64 positions, or the mixed form's fixed-point words (fix_diff)
  const double xi = MIXED ? 0.0 : a.x[i], yi = MIXED ? 0.0 : a.y[i], zi = MIXED ? 0.0 : a.z[i];
  const uint32_t uxi = MIXED ? a.ux[i] : 0u, uyi = MIXED ? a.uy[i] : 0u, uzi = MIXED ? a.uz[i] : 0u;
  const long long hb[3] = {half_bits(a.box[0]), half_bits(a.box[1]), half_bits(a.box[2])};
  const double* rho = a.rho + (a.rho_per_rep ? (long long)r * a.N : 0);
  const double rc2 = a.rc * a.rc;
  double part = 0.0;
  for (int k0 = 0; k0 < cnt; k0 += 32 * MCW_SLOTS) {
    int jv[MCW_SLOTS];
    bool in[MCW_SLOTS];
#pragma unroll
    for (int u = 0; u < MCW_SLOTS; ++u) {
      const int k = k0 + lane + 32 * u;
      in[u] = k < cnt;
      jv[u] = in[u] ? row[k] : i;
    }
    int tj[MCW_SLOTS];
    double xj[MCW_SLOTS], yj[MCW_SLOTS], zj[MCW_SLOTS], rj[MCW_SLOTS];
    uint32_t uxj[MCW_SLOTS], uyj[MCW_SLOTS], uzj[MCW_SLOTS];
#pragma unroll
    for (int u = 0; u < MCW_SLOTS; ++u) {
      tj[u] = ty[jv[u]];
      if constexpr (MIXED) {
        uxj[u] = a.ux[jv[u]];
        uyj[u] = a.uy[jv[u]];
        uzj[u] = a.uz[jv[u]];
      } else {
        xj[u] = a.x[jv[u]];
        yj[u] = a.y[jv[u]];
        zj[u] = a.z[jv[u]];
      }
      rj[u] = REEMBED ? rho[jv[u]] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < MCW_SLOTS; ++u) {
      if (!in[u]) continue;
      double vp, vm, fp = 0.0, fm = 0.0;
      if constexpr (MIXED) {
        // FP32 distance and table values, FP64 differences and sums
        const float dx = fix_diff(uxj[u], uxi, a.ul[0]);
        const float dy = fix_diff(uyj[u], uyi, a.ul[1]);
        const float dz = fix_diff(uzj[u], uzi, a.ul[2]);
        const float r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= (float)rc2) continue;
        float tt;
        const int jj = spline32_locate(a.tab32.sp[0], sqrtf(r2), tt, err);
        vp = (double)spline32_val_at(a.tab32.sp[tp + tj[u]], jj, tt);
        vm = (double)spline32_val_at(a.tab32.sp[t + tj[u]], jj, tt);
        if (REEMBED) {
          fp = (double)spline32_val_at(a.tab32.sp[3 + tp], jj, tt);
          fm = (double)spline32_val_at(a.tab32.sp[3 + t], jj, tt);
        }
      } else {
        const double dx = mimg_w(xj[u] - xi, a.box[0], hb[0]);
        const double dy = mimg_w(yj[u] - yi, a.box[1], hb[1]);
        const double dz = mimg_w(zj[u] - zi, a.box[2], hb[2]);
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= rc2) continue;
        double tt;
        const int jj = spline_locate(a.tab.sp[0], r2 * rsqrt_nr(r2), tt, err);
        vp = spline_val_at(a.tab.sp[tp + tj[u]], jj, tt);
        vm = spline_val_at(a.tab.sp[t + tj[u]], jj, tt);
        if (REEMBED) {
          fp = spline_val_at(a.tab.sp[3 + tp], jj, tt);
          fm = spline_val_at(a.tab.sp[3 + t], jj, tt);
        }
      }
      part += vp - vm;
      if constexpr (REEMBED) {
        const double drho = fp - fm;
        part += spline_val(a.tab.sp[5 + tj[u]], rj[u] + drho, err) - spline_val(a.tab.sp[5 + tj[u]], rj[u], err);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  double own;
  if constexpr (REEMBED) {
    const double ri = rho[i];
    own = spline_val(a.tab.sp[5 + tp], ri, err) - spline_val(a.tab.sp[5 + t], ri, err);
  } else {
    own = t ? -a.dF[i] : a.dF[i];
  }
  return part + own;
}

template <int BLOCK>
__device__ __forceinline__ void block_reduce3(int& a, int& b, double& c) {
  __shared__ int sa[BLOCK / 32], sb[BLOCK / 32];
  __shared__ double sc[BLOCK / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sa[w] = a; sb[w] = b; sc[w] = c; }
  __syncthreads();
  if (w == 0) {
    a = l < BLOCK / 32 ? sa[l] : 0;
    b = l < BLOCK / 32 ? sb[l] : 0;
    c = l < BLOCK / 32 ? sc[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
      c += __shfl_xor_sync(0xffffffffu, c, o);
    }
  }
}

__device__ __forceinline__ int draw_colour(const McArgs& a, uint2 key, long long step, uint64_t* ug53) {
  const uint4 w = philox4x32_10(make_uint4((uint32_t)step, (uint32_t)((uint64_t)step >> 32), 0xFFFFFFFFu, TAG_STEP), key);
  if (ug53) *ug53 = top53(w.z, w.w);
  return (int)below64(w.x, w.y, (uint64_t)a.n_colours);
}

// Screened form of the shell dE with re-embedding (a.screen).  With
// species-dependent densities a trial's dE holds 2 x 58 + 2 embedding
// evaluations, which in FP64 (a small share of GB300's arithmetic) bound the
// step.  The local decision is taken instead on this FP32 dE: the pair part
// in FP64 as in delta_e (exact in arithmetic) rounded once, the own and the
// neighbours' embedding changes in FP32 from the per-site floats (rho, and
// F32_t(rho) cached).  *err bounds its distance from the FP64 dE: emb_err per
// evaluation (the bound of screen.h), 2^-18 of the sum of |terms| for the
// float additions and 2^-21 of the sizes of the final sums.  *in is false
// when an argument left [emb_lo, emb_hi].
__device__ float delta_e_screen(const McArgs& a, int r, int i, int t, float* err, bool* in) {
  const uint8_t* ty = a.types + (long long)r * a.N;
  const int* row = a.nbr + (long long)i * a.K;
  const float2* rf = a.rf + (long long)r * a.N;
  const int S = a.n_shells;
  double pair = a.shell_tab[0];
  float re = 0.0f, ab = 0.0f;
  bool ok = true;
  int k = 0;
  for (int s = 0; s < S; ++s) {
    const float dfs = (float)a.shell_tab[1 + S + s];
    const float drho = t ? -dfs : dfs;
    const int end = a.shell_end[s];
    int cnt = 0;
#pragma unroll 4
    for (; k < end; ++k) {
      const int j = row[k];
      const int tj = ty[j];
      const float2 v = rf[j];
      cnt += tj;
      const float x1 = v.x + drho;
      ok &= emb32_in(a, v.x) & emb32_in(a, x1);
      const float d = emb32_val(a, tj, x1) - v.y;
      re += d;
      ab += fabsf(d);
    }
    pair = fma((double)cnt, a.shell_tab[1 + s], pair);
  }
  if (t) pair = -pair;
  const float2 ri = rf[i];
  ok &= emb32_in(a, ri.x);
  const float own = emb32_val(a, 1 - t, ri.x) - ri.y;
  const float p32 = (float)pair;
  *in = ok;
  *err = fmaf((float)(2 * k + 2), a.emb_err,
              fmaf(3.814697265625e-06f, ab, 4.76837158203125e-07f * (fabsf(p32) + fabsf(own) + fabsf(re))));
  return (p32 + own) + re;
}

// lane's share of the FP64 shell dE with re-embedding of site i (species t):
// neighbours k = lane, lane + 32, ... (their B-count pair terms and
// re-embeddings); lane 0 adds the constant and the own change.  The warp's
// sum is delta_e<true, true> up to the order of the additions.
__device__ double delta_e_shell_lane(const McArgs& a, int r, int i, int t, int lane, unsigned* err) {
  const uint8_t* ty = a.types + (long long)r * a.N;
  const int* row = a.nbr + (long long)i * a.K;
  const double* rho = a.rho + (a.rho_per_rep ? (long long)r * a.N : 0);
  const int S = a.n_shells;
  const int n = a.shell_end[S - 1];
  const double sg = t ? -1.0 : 1.0;
  double v = 0.0;
  for (int k = lane; k < n; k += 32) {
    int s = 0;
    while (k >= a.shell_end[s]) ++s;
    const int j = row[k];
    const int tj = ty[j];
    const double drho = sg * a.shell_tab[1 + S + s];
    const double rj = rho[j];
    v += sg * (double)tj * a.shell_tab[1 + s];
    v += spline_val(a.tab.sp[5 + tj], rj + drho, err) - spline_val(a.tab.sp[5 + tj], rj, err);
  }
  if (lane == 0) {
    const double ri = rho[i];
    v += sg * a.shell_tab[0] + spline_val(a.tab.sp[6 - t], ri, err) - spline_val(a.tab.sp[5 + t], ri, err);
  }
  return v;
}

template <bool SHELL, bool REEMBED>
__global__ void __launch_bounds__(MC_BLOCK) k_propose(McArgs a) {
  const int r = blockIdx.y;
  const RepParams p = a.rp[r];
  const long long step = a.rs[r].step;
  const int c = draw_colour(a, p.key, step, nullptr);
  const int d0 = a.col_start[c];
  const int D = a.col_start[c + 1] - d0;
  const int d = blockIdx.x * MC_BLOCK + threadIdx.x;
  int dn = 0, acc = 0, tie = 0, site = -1, t = 0, dec = 0;
  uint64_t u53 = 0;
  double sde = 0.0;
  if (d < D) {
    const int g = d0 + d;
    const int base = a.dom_start[g];
    const int size = a.dom_start[g + 1] - base;
    if (size > 0) {
      const uint4 w = philox4x32_10(make_uint4((uint32_t)step, (uint32_t)((uint64_t)step >> 32), (uint32_t)d, TAG_TRIAL), p.key);
      site = a.dom_sites[base + pick_index(a.pick, w.x, w.y, size)];
      u53 = top53(w.z, w.w);
      t = a.types[(long long)r * a.N + site];
      const double sg = t ? -1.0 : 1.0;
      bool screened = false;
      if constexpr (SHELL && REEMBED) {
        if (a.screen) {
          screened = true;
          float err;
          bool in;
          const float e32 = delta_e_screen(a, r, site, t, &err, &in);
          const float cm = (float)(sg * p.dmu0), b32 = (float)p.beta;
          const float x32 = b32 * (e32 + cm);
          const float dx = b32 * fmaf(4.76837158203125e-07f, fabsf(e32) + fabsf(cm), err) * 1.0001f +
                           fabsf(x32) * 4.76837158203125e-07f;
          dec = in ? screen32(x32, dx, u53) : -1;
          if (dec > 0) {
            acc = 1;
            dn = t ? -1 : 1;
          }
        }
      }
      if (!screened) {
        const double de = delta_e<SHELL, REEMBED>(a, r, site, a.err);
        if (!isfinite(de)) atomicOr(a.err, ERRF_NONFINITE);
        const double X = p.beta * fma(sg, p.dmu0, de);
        if (metropolis(X, u53, &tie)) {
          acc = 1;
          dn = t ? -1 : 1;
          sde = de;
        }
      }
    }
  }
  const int lane = threadIdx.x & 31;
  if constexpr (SHELL && REEMBED) {
    // trials the screen left open: FP64 dE by the whole warp, one at a time
    // (the energy of the screened form is not tracked: no dE sum)
    unsigned open = __ballot_sync(0xffffffffu, dec < 0);
    while (open) {
      const int src = __ffs(open) - 1;
      open &= open - 1u;
      const int si = __shfl_sync(0xffffffffu, site, src), st = __shfl_sync(0xffffffffu, t, src);
      double v = delta_e_shell_lane(a, r, si, st, lane, a.err);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == src) {
        if (!isfinite(v)) atomicOr(a.err, ERRF_NONFINITE);
        const double X = p.beta * fma(t ? -1.0 : 1.0, p.dmu0, v);
        if (metropolis(X, u53, &tie)) {
          acc = 1;
          dn = t ? -1 : 1;
        }
      }
    }
  }
  // compact the accepted sites: warp ballot, one reservation per warp
  const unsigned m = __ballot_sync(0xffffffffu, acc);
  int slot_base = 0;
  if (m) {
    if (lane == 0) slot_base = atomicAdd(&a.acc[r].nacc, __popc(m));
    slot_base = __shfl_sync(0xffffffffu, slot_base, 0);
    if (acc) a.acc_list[(long long)r * a.dmax + slot_base + __popc(m & ((1u << lane) - 1u))] = site | (t << 30);
  }
  if (tie) atomicAdd(&a.acc[r].ties, 1);
  int dummy = 0;
  block_reduce3<MC_BLOCK>(dn, dummy, sde);
  if (threadIdx.x == 0 && (dn != 0 || sde != 0.0)) {
    atomicAdd(&a.acc[r].dn, dn);
    atomicAdd(&a.acc[r].sum_de, sde);
  }
}

// General form: one warp per trial.  Same draws and rule as k_propose.
// One trial (one warp) per block: a colour step of a nanocrystal holds a
// few hundred to a few thousand trials, and single-warp blocks spread them
// over every SM (four-warp blocks left the 343 trials of a 17 nm cell on 86
// SMs, and up to 12 of the 1,331 of a 25 nm cell on one SM against 9).
constexpr int MCW_BLOCK = 32;

template <bool REEMBED, bool MIXED>
__global__ void __launch_bounds__(MCW_BLOCK) k_propose_warp(McArgs a) {
  const int r = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int d = blockIdx.x * (MCW_BLOCK / 32) + (threadIdx.x >> 5);
  const RepParams p = a.rp[r];
  const long long step = a.rs[r].step;
  const int c = draw_colour(a, p.key, step, nullptr);
  const int d0 = a.col_start[c];
  const int D = a.col_start[c + 1] - d0;
  if (d >= D) return;
  const int g = d0 + d;
  const int base = a.dom_start[g];
  const int size = a.dom_start[g + 1] - base;
  if (size == 0) return;
  const uint4 w = philox4x32_10(make_uint4((uint32_t)step, (uint32_t)((uint64_t)step >> 32), (uint32_t)d, TAG_TRIAL), p.key);
  const int site = a.dom_sites[base + pick_index(a.pick, w.x, w.y, size)];
  const double de = delta_e_warp<REEMBED, MIXED>(a, r, site, lane, a.err);
  if (lane != 0) return;
  const int t = a.types[(long long)r * a.N + site];
  if (!isfinite(de)) atomicOr(a.err, ERRF_NONFINITE);
  int tie = 0;
  const double X = p.beta * fma(t ? -1.0 : 1.0, p.dmu0, de);
  if (metropolis(X, top53(w.z, w.w), &tie)) {
    const int slot = atomicAdd(&a.acc[r].nacc, 1);
    a.acc_list[(long long)r * a.dmax + slot] = site | (t << 30);
    atomicAdd(&a.acc[r].dn, t ? -1 : 1);
    atomicAdd(&a.acc[r].sum_de, de);
  }
  if (tie) atomicAdd(&a.acc[r].ties, 1);
}

// flip site i of replica r and scatter its density change to its neighbours
// (no two sites of one colour share a neighbour: they are > 2 r_c apart)
template <bool SHELL, bool REEMBED>
__device__ void commit_site(const McArgs& a, int r, int i, unsigned* err) {
  uint8_t* ty = a.types + (long long)r * a.N;
  const int t = ty[i];
  ty[i] = (uint8_t)(1 - t);
  if (a.vel[0] && r == 0) {
    const double f = sqrt(a.mass[t] / a.mass[1 - t]);
    a.vel[0][i] *= f;
    a.vel[1][i] *= f;
    a.vel[2][i] *= f;
  }
  if constexpr (REEMBED) {
    const int* row = a.nbr + (long long)i * a.K;
    double* rho = a.rho + (a.rho_per_rep ? (long long)r * a.N : 0);
    if constexpr (SHELL) {
      const int S = a.n_shells;
      int k = 0;
      float2* rf = a.screen ? a.rf + (long long)r * a.N : nullptr;
      for (int s = 0; s < S; ++s) {
        const double dfs = a.shell_tab[1 + S + s];
        const double drho = t ? -dfs : dfs;
        for (; k < a.shell_end[s]; ++k) {
          const int j = row[k];
          const double nr = rho[j] + drho;
          rho[j] = nr;
          if (rf) {
            // the screened form's float copy and its FP32 embedding value
            const float r32 = (float)nr;
            rf[j] = make_float2(r32, emb32_val(a, ty[j], r32));
          }
        }
      }
      if (rf) rf[i].y = emb32_val(a, 1 - t, rf[i].x);
    } else {
      const int cnt = a.nbr_cnt[i];
      const int tp = 1 - t;
      const long long hb[3] = {half_bits(a.box[0]), half_bits(a.box[1]), half_bits(a.box[2])};
      for (int k = 0; k < cnt; ++k) {
        const int j = row[k];
        const double dx = mimg_w(a.x[j] - a.x[i], a.box[0], hb[0]);
        const double dy = mimg_w(a.y[j] - a.y[i], a.box[1], hb[1]);
        const double dz = mimg_w(a.z[j] - a.z[i], a.box[2], hb[2]);
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= a.rc * a.rc) continue;
        if (a.mixed) {
          float tt;
          const int jj = spline32_locate(a.tab32.sp[3], sqrtf((float)r2), tt, err);
          rho[j] += (double)spline32_val_at(a.tab32.sp[3 + tp], jj, tt) -
                    (double)spline32_val_at(a.tab32.sp[3 + t], jj, tt);
        } else {
          double tt;
          const int jj = spline_locate(a.tab.sp[3], r2 * rsqrt_nr(r2), tt, err);
          rho[j] += spline_val_at(a.tab.sp[3 + tp], jj, tt) - spline_val_at(a.tab.sp[3 + t], jj, tt);
        }
      }
    }
  }
}

// item k of an accepted flip of site i (old species t) on the rigid lattice
// with re-embedding: k < n, neighbour k's density change (and the screened
// form's floats there); k = n, the site's species (and its FP32 embedding
// value).  No two items touch a common site: the accepts of one colour are
// more than 2 r_c apart.
__device__ __forceinline__ void commit_item_shell(const McArgs& a, int r, int i, int t, int k, int n) {
  uint8_t* ty = a.types + (long long)r * a.N;
  float2* rf = a.screen ? a.rf + (long long)r * a.N : nullptr;
  if (k < n) {
    int s = 0;
    while (k >= a.shell_end[s]) ++s;
    const double dfs = a.shell_tab[1 + a.n_shells + s];
    const int j = a.nbr[(long long)i * a.K + k];
    double* rho = a.rho + (a.rho_per_rep ? (long long)r * a.N : 0);
    const double nr = rho[j] + (t ? -dfs : dfs);
    rho[j] = nr;
    if (rf) {
      const float r32 = (float)nr;
      rf[j] = make_float2(r32, emb32_val(a, ty[j], r32));
    }
  } else {
    ty[i] = (uint8_t)(1 - t);
    if (a.vel[0] && r == 0) {
      const double f = sqrt(a.mass[t] / a.mass[1 - t]);
      a.vel[0][i] *= f;
      a.vel[1][i] *= f;
      a.vel[2][i] *= f;
    }
    if (rf) rf[i].y = emb32_val(a, 1 - t, rf[i].x);
  }
}

template <bool SHELL, bool REEMBED>
__global__ void __launch_bounds__(MC_BLOCK) k_commit(McArgs a) {
  const int r = blockIdx.y;
  StepAcc* A = &a.acc[r];
  RepState* S = &a.rs[r];
  const RepParams p = a.rp[r];
  const int nacc = *(volatile int*)&A->nacc;
  const int dn = *(volatile int*)&A->dn;
  const long long n = S->n;
  const long long step = S->step;
  uint64_t ug53;
  const int c = draw_colour(a, p.key, step, &ug53);
  bool G = false;
  int tie = 0;
  if (nacc > 0) {
    const double Y = p.beta * p.kappa_p * (double)dn * ((double)dn + 2.0 * ((double)n - p.n0));
    G = metropolis(Y, ug53, &tie);
  }
  if (G) {
    if constexpr (SHELL && REEMBED) {
      // one thread per (accept, neighbour) and one per accepted site: the
      // density change (and the screened form's floats) of each neighbour,
      // then the species.  The old species travels in the list entry, so
      // no thread reads a species another thread of this launch writes.
      const int n = a.shell_end[a.n_shells - 1];
      const int items = nacc * (n + 1);
      for (int it = blockIdx.x * MC_BLOCK + threadIdx.x; it < items; it += gridDim.x * MC_BLOCK) {
        const int q = it / (n + 1), k = it - q * (n + 1);
        const int e = a.acc_list[(long long)r * a.dmax + q];
        const int i = e & 0x3FFFFFFF, t = e >> 30;
        commit_item_shell(a, r, i, t, k, n);
      }
    } else {
      for (int q = blockIdx.x * MC_BLOCK + threadIdx.x; q < nacc; q += gridDim.x * MC_BLOCK)
        commit_site<SHELL, REEMBED>(a, r, a.acc_list[(long long)r * a.dmax + q] & 0x3FFFFFFF, a.err);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned ticket = atomicAdd(&A->done, 1u);
    if (ticket == gridDim.x - 1) {
      __threadfence();
      const int D = a.col_start[c + 1] - a.col_start[c];
      S->trials += D;
      S->local_acc += nacc;
      S->near_ties += *(volatile int*)&A->ties + tie;
      long long nn = n;
      if (nacc > 0) {
        S->global_trials += 1;
        if (G) {
          S->global_acc += 1;
          S->flips += nacc;
          nn = n + dn;
          S->n = nn;
          S->energy += *(volatile double*)&A->sum_de;
        }
      }
      const double cc = (double)nn / (double)a.N;
      S->sum_c += cc;
      S->sum_c2 += cc * cc;
      S->steps += 1;
      S->step = step + 1;
      A->dn = 0;
      A->nacc = 0;
      A->sum_de = 0.0;
      A->ties = 0;
      __threadfence();
      A->done = 0u;
    }
  }
}

// the screened form's per-site floats of replica r from its densities
__global__ void k_fill_rf(McArgs a, int r) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  const float r32 = (float)a.rho[(long long)r * a.N + i];
  a.rf[(long long)r * a.N + i] = make_float2(r32, emb32_val(a, a.types[(long long)r * a.N + i], r32));
}

void launch_fill_rf(const McArgs& a, int r, cudaStream_t st) {
  k_fill_rf<<<(unsigned)((a.N + 255) / 256), 256, 0, st>>>(a, r);
}

// dE of a list of sites with the sweep's own device function (general
// form: one warp per site, as in the sweep)
template <bool SHELL, bool REEMBED>
__global__ void k_delta_e_list(McArgs a, int r, const int* sites, int n, double* out) {
  if (SHELL) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) out[q] = delta_e<SHELL, REEMBED>(a, r, sites[q], a.err);
  } else {
    const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= n) return;
    const double de = a.mixed ? delta_e_warp<REEMBED, true>(a, r, sites[q], threadIdx.x & 31, a.err)
                              : delta_e_warp<REEMBED, false>(a, r, sites[q], threadIdx.x & 31, a.err);
    if ((threadIdx.x & 31) == 0) out[q] = de;
  }
}

// ----------------------------------------------------------------- launch
template <bool SHELL, bool REEMBED>
static void launch_step_t(const McArgs& a, cudaStream_t st, int phase) {
  const int cb = (a.dmax + MC_BLOCK - 1) / MC_BLOCK;
  if (phase != 2) {
    if (SHELL) {
      k_propose<SHELL, REEMBED><<<dim3(cb, a.R), MC_BLOCK, 0, st>>>(a);
    } else {
      const int wb = (a.dmax + MCW_BLOCK / 32 - 1) / (MCW_BLOCK / 32);
      if (a.mixed) k_propose_warp<REEMBED, true><<<dim3(wb, a.R), MCW_BLOCK, 0, st>>>(a);
      else k_propose_warp<REEMBED, false><<<dim3(wb, a.R), MCW_BLOCK, 0, st>>>(a);
    }
  }
  // the rigid re-embedding commit runs one thread per (accept, neighbour):
  // as many blocks as the propose
  if (phase != 1) k_commit<SHELL, REEMBED><<<dim3((SHELL && REEMBED) ? cb : (cb < 8 ? cb : 8), a.R), MC_BLOCK, 0, st>>>(a);
}

void launch_colour_step(const McArgs& a, bool shell, bool reembed, cudaStream_t st, int phase) {
  if (shell) {
    if (reembed) launch_step_t<true, true>(a, st, phase);
    else launch_step_t<true, false>(a, st, phase);
  } else {
    if (reembed) launch_step_t<false, true>(a, st, phase);
    else launch_step_t<false, false>(a, st, phase);
  }
}

void launch_delta_e_list(const McArgs& a, bool shell, bool reembed, int r, const int* sites, int n,
                         double* out, cudaStream_t st) {
  const int b = 128, g = shell ? (n + b - 1) / b : (n + 3) / 4;
  if (g == 0) return;
  if (shell) {
    if (reembed) k_delta_e_list<true, true><<<g, b, 0, st>>>(a, r, sites, n, out);
    else k_delta_e_list<true, false><<<g, b, 0, st>>>(a, r, sites, n, out);
  } else {
    if (reembed) k_delta_e_list<false, true><<<g, b, 0, st>>>(a, r, sites, n, out);
    else k_delta_e_list<false, false><<<g, b, 0, st>>>(a, r, sites, n, out);
  }
}

}  // namespace vcsgc
