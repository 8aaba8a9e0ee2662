// lattice.cuh -- device helpers of the fused rigid-lattice colour step shared
// by its per-step launch (kernels_lattice.cu) and its cluster-resident form
// (kernels_cluster.cu): site decode, the effective species of a bit-packed
// word, the compile-time five-shell BCC rows, and the local and global
// decisions of the composite move (Sec. III B 2, Eqs. trans_vcsgc_par1/par2).
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace vcsgc {

// n / d for 0 <= n < 2^22 by a float reciprocal and one correction: the
// float quotient is within 2^-23 relative of n/d < 2^22, so off by at most 1
__device__ __forceinline__ int fdiv(int n, int d, float rcp) {
  int q = __float2int_rz(__int2float_rn(n) * rcp);
  const int r = n - q * d;
  q += (r < 0) ? -1 : (r >= d ? 1 : 0);
  return q;
}

// effective 32 species bits of a word under the pending decision mask gm
__device__ __forceinline__ uint32_t eff32(unsigned long long w, uint32_t gm) {
  return (uint32_t)w ^ ((uint32_t)(w >> 32) & gm);
}

// The five-shell BCC neighbourhood (r_c between sqrt(3) a and 2 a: half-
// lattice offsets with |h|^2 in {3, 4, 8, 11, 12}, 58 sites) as compile-time
// rows.  For basis b and row q: bits 7s..7s+6 hold the 7-bit window mask of
// shell s (window bit h_x + 3), bits 40..43 hold dy + 2 and bits 44..47
// dz + 2.  Rows and masks are the ones the host derives from the sorted
// offset table; the host compares the two before it selects this form.  As
// constants the masks let the compiler drop the (row, shell) pairs that
// hold no site (33 of the 65 are non-empty) and turn one-bit masks into
// bit tests.
__host__ __device__ __forceinline__ constexpr unsigned long long bcc5_row(int b, int q) {
  switch (16 * b + q) {
    case 0: return 0x110228220014ull;
    case 1: return 0x210008288414ull;
    case 2: return 0x120008288414ull;
    case 3: return 0x220008201114ull;
    case 4: return 0x320002888400ull;
    case 5: return 0x230002888400ull;
    case 6: return 0x310222820000ull;
    case 7: return 0x130222820000ull;
    case 8: return 0x330220020000ull;
    case 9: return 0x100002800000ull;
    case 10: return 0x200002800000ull;
    case 11: return 0x010002800000ull;
    case 12: return 0x020002800000ull;
    case 16: return 0x220008201114ull;
    case 17: return 0x320008288414ull;
    case 18: return 0x230008288414ull;
    case 19: return 0x330228220014ull;
    case 20: return 0x210002888400ull;
    case 21: return 0x120002888400ull;
    case 22: return 0x110220020000ull;
    case 23: return 0x310222820000ull;
    case 24: return 0x130222820000ull;
    case 25: return 0x420002800000ull;
    case 26: return 0x430002800000ull;
    case 27: return 0x240002800000ull;
    case 28: return 0x340002800000ull;
    default: return 0ull;
  }
}

__device__ __forceinline__ int wrap_add(int y, int dy, int n) {
  y += dy;
  return y < 0 ? y + n : (y >= n ? y - n : y);
}

// dE of flipping the site (FP64): the A->B value C + sum_s b_s G_s + dF_i,
// negated for B->A (i is the site index within its replica)
template <int NS>
__device__ __forceinline__ double lattice_de64(const LatArgs& a, const int (&cnt)[NS], int i, int t) {
  double de = a.C;
#pragma unroll
  for (int s = 0; s < NS; ++s) de = fma((double)cnt[s], a.G[s], de);
  de += a.df_uniform ? a.dF0 : a.dF[i];
  return t ? -de : de;
}

// Local Metropolis decision of trial site i, identical to the FP64 decision
// u < min{1, exp(-X)}, X = beta (dE + s dmu0).  X is first formed in FP32
// from the integer counts: X32 = +-beta (C + dmu0 + sum_s b_s G_s + dF_i).
// lr.dx bounds |X32 - X| (FP32 rounding of each input and partial sum,
// derived on the host from the magnitudes of the terms); only when X32 and
// that bound cannot settle the decision is X recomputed in FP64 (rare).
template <int NS>
__device__ __forceinline__ bool lattice_accept(const LatArgs& a, const LatRep& lr, const RepParams& p,
                                               const int (&cnt)[NS], int i, int t, uint64_t u53,
                                               int* tie) {
  float s32 = lr.cpd32;
#pragma unroll
  for (int s = 0; s < NS; ++s) s32 = fmaf((float)cnt[s], a.G32[s], s32);
  s32 += a.df_uniform ? 0.0f : a.dF32[i];
  const float x32 = (t ? -lr.beta32 : lr.beta32) * s32;
  if (!isfinite(x32)) atomicOr(a.err, ERRF_NONFINITE);
  const float dx = lr.dx + fabsf(x32) * 4.76837158203125e-07f;  // + |X| 2^-21
  const int dec = screen32(x32, dx, u53);
  if (dec >= 0) return dec != 0;
  const double de = lattice_de64<NS>(a, cnt, i, t);
  const double sg = t ? -1.0 : 1.0;
  return metropolis(p.beta * fma(sg, p.dmu0, de), u53, tie);
}

// Global decision of a step with dn != 0 accepted locally out of n at its
// start: u_g < min{1, exp(-Y)}, Y = beta kappa_p dn (dn + 2 (n - n0))
// (Eq. trans_vcsgc_par2), identical to the FP64 decision: Y is formed in FP32
// with a bound on its rounding (beta kappa_p and n0 rounded to float, n <
// 2^24 exact, two products and two sums), FP64 only when the screen cannot
// settle it or |Y| is tiny.
__device__ __forceinline__ bool global_accept(const LatRep& lr, const RepParams& p, int dn, long long n,
                                              uint64_t ug53, int* tie) {
  if (dn == 0) {
    if (ug53 >= U53_NEAR_ONE) *tie = 1;
    return true;
  }
  const float fdn = (float)dn, diff = (float)n - lr.n0_32;
  const float y32 = lr.bk32 * fdn * fmaf(2.0f, diff, fdn);
  const float dy = fabsf(lr.bk32 * fdn) * (fabsf(fdn) + 2.0f * ((float)n + lr.n0_32)) * 4.76837158203125e-07f;
  if (fabsf(y32) > 1e-6f) {
    const int dec = screen32(y32, dy, ug53);
    if (dec >= 0) return dec != 0;
  }
  const double Y = p.beta * p.kappa_p * (double)dn * ((double)dn + 2.0 * ((double)n - p.n0));
  return metropolis(Y, ug53, tie);
}

__device__ __forceinline__ int lat_colour(const LatArgs& a, uint2 key, long long step, uint64_t* ug53) {
  const uint4 w = philox4x32_10(make_uint4((uint32_t)step, (uint32_t)((uint64_t)step >> 32), 0xFFFFFFFFu, TAG_STEP), key);
  if (ug53) *ug53 = top53(w.z, w.w);
  return (int)below64(w.x, w.y, (uint64_t)a.n_colours);
}

}  // namespace vcsgc
