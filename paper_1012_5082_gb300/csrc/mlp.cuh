// mlp.cuh -- device pieces of the delayed-acceptance surrogate shared by the
// colour step (inference, one trial per lane) and the training kernels.
//
// Network: ten environment counts c (own B counts in shells 1-5, then the
// first-shell neighbours' summed B counts in shells 1-5) scaled to
// x = c / max_c, then z1 = W1 x + b1, h1 = SiLU(z1), z2 = W2 h1 + b2,
// h2 = SiLU(z2), g = w3 . h2 + b3 (g predicts E(site = B) - E(site = A)).
// SiLU(z) = z (1 + tanh(z / 2)) / 2 with the hardware tanh.
//
// Tensor-core form: a warp evaluates a tile of 16 samples with mma.sync
// m16n8k16 (BF16 operands, FP32 accumulation).  The inputs are padded from
// 10 to 16 columns; layer 1 is 8 MMAs (n = 64 outputs in 8 tiles of 8),
// layer 2 is 32 (k = 64 in 4 tiles of 16).  The accumulator fragments of
// layer 1 are re-packed in registers as the A fragments of layer 2 (the two
// layouts coincide), so h1 never leaves the registers.  The output layer is
// an FP32 dot product reduced over the four lanes of each row.
//
// Weights enter as pre-packed fragments (each lane's two B registers of
// every MMA, 256 bytes per warp-wide load), produced from the FP32 master
// parameters by k_mlp_pack.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace vcsgc {

constexpr int MLP_IN = 10;
constexpr int MLP_H = 64;
constexpr int MLP_OFF_W1 = 0;
constexpr int MLP_OFF_B1 = MLP_OFF_W1 + MLP_H * MLP_IN;
constexpr int MLP_OFF_W2 = MLP_OFF_B1 + MLP_H;
constexpr int MLP_OFF_B2 = MLP_OFF_W2 + MLP_H * MLP_H;
constexpr int MLP_OFF_W3 = MLP_OFF_B2 + MLP_H;
constexpr int MLP_OFF_B3 = MLP_OFF_W3 + MLP_H;
constexpr int MLP_NPARAM = MLP_OFF_B3 + 1;  // 4929
// packed fragments (uint2 per lane): W1 as layer-1 B [8 n-tiles], W2 as
// layer-2 B [8 n][4 k], W2 transposed as the B of the back-propagation
// product d2 W2 [8 n][4 k]; vec = b1 | b2 | w3 | b3 (FP32)
constexpr int MLP_W1F = 8 * 32;
constexpr int MLP_W2F = 8 * 4 * 32;
constexpr int MLP_VEC = 3 * MLP_H + 4;

struct MlpW {
  const uint2* w1f;
  const uint2* w2f;
  const uint2* w2tf;
  const float* vec;
};

// 1 / max_c: the counts when every site is B on the BCC lattice
__device__ __forceinline__ float mlp_in_scale(int c) {
  switch (c) {
    case 0: return 1.0f / 8.0f;
    case 1: return 1.0f / 6.0f;
    case 2: return 1.0f / 12.0f;
    case 3: return 1.0f / 24.0f;
    case 4: return 1.0f / 8.0f;
    case 5: return 1.0f / 56.0f;
    case 6: return 1.0f / 48.0f;
    case 7: return 1.0f / 96.0f;
    case 8: return 1.0f / 192.0f;
    default: return 1.0f / 64.0f;
  }
}

__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x = lo (low half)
  return *reinterpret_cast<const uint32_t*>(&v);
}

// The ten scaled descriptor inputs as BF16 pairs (p[4] = inputs 8, 9): own
// B counts in shells 1-5, then the first-shell neighbours' summed counts
__device__ __forceinline__ void mlp_pairs(const int (&own)[5], const int (&nb)[5], uint32_t (&p)[5]) {
  float x[10];
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    x[s] = (float)own[s] * mlp_in_scale(s);
    x[5 + s] = (float)nb[s] * mlp_in_scale(5 + s);
  }
#pragma unroll
  for (int c = 0; c < 5; ++c) p[c] = bf16x2(x[2 * c], x[2 * c + 1]);
}

// D += A (16x16, row) * B (16x8, col); BF16 operands, FP32 accumulators
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint2 b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b.x), "r"(b.y));
}

// SiLU through the hardware tanh: sigma(z) = (1 + tanh(z / 2)) / 2
__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sigm(float z) { return fmaf(0.5f, tanh_fast(0.5f * z), 0.5f); }
// sigma of two values (FP32 tanh.approx each)
__device__ __forceinline__ void sigm2(float za, float zb, float& sa, float& sb) {
  sa = sigm(za);
  sb = sigm(zb);
}
__device__ __forceinline__ void silu2(float za, float zb, float& ya, float& yb) {
  float sa, sb;
  sigm2(za, zb, sa, sb);
  ya = za * sa;
  yb = zb * sb;
}
// BF16 pair (SiLU(za), SiLU(zb)), za in the low half
__device__ __forceinline__ uint32_t silu_bf16x2(float za, float zb) {
  float ya, yb;
  silu2(za, zb, ya, yb);
  return bf16x2(ya, yb);
}
// d SiLU / dz = sigma (1 + z (1 - sigma))
__device__ __forceinline__ float dsilu(float z) {
  const float s = sigm(z);
  return s * fmaf(z, 1.0f - s, 1.0f);
}

// Forward pass of one 16-sample tile held as the A fragment (x0..x3) of the
// scaled inputs.  z1, z2: pre-activations in accumulator layout (n-tile,
// value); y_lo / y_hi: outputs of rows g and g + 8 (g = lane / 4), valid in
// every lane.
__device__ __forceinline__ void mlp_tile_forward(const MlpW& w, uint32_t x0, uint32_t x1, uint32_t x2,
                                                 uint32_t x3, float (&z1)[8][4], float (&z2)[8][4],
                                                 float& y_lo, float& y_hi) {
  const int lane = threadIdx.x & 31, t = lane & 3;
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    const float2 bb = __ldg(reinterpret_cast<const float2*>(w.vec) + 4 * n + t);  // b1[8n + 2t], +1
    z1[n][0] = bb.x;
    z1[n][1] = bb.y;
    z1[n][2] = bb.x;
    z1[n][3] = bb.y;
    mma_bf16(z1[n], x0, x1, x2, x3, __ldg(w.w1f + n * 32 + lane));
  }
  uint32_t h[4][4];  // layer-2 A fragments, k-tile kk
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    h[kk][0] = silu_bf16x2(z1[2 * kk][0], z1[2 * kk][1]);
    h[kk][1] = silu_bf16x2(z1[2 * kk][2], z1[2 * kk][3]);
    h[kk][2] = silu_bf16x2(z1[2 * kk + 1][0], z1[2 * kk + 1][1]);
    h[kk][3] = silu_bf16x2(z1[2 * kk + 1][2], z1[2 * kk + 1][3]);
  }
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    const float2 bb = __ldg(reinterpret_cast<const float2*>(w.vec + MLP_H) + 4 * n + t);  // b2
    z2[n][0] = bb.x;
    z2[n][1] = bb.y;
    z2[n][2] = bb.x;
    z2[n][3] = bb.y;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
      mma_bf16(z2[n], h[kk][0], h[kk][1], h[kk][2], h[kk][3], __ldg(w.w2f + (n * 4 + kk) * 32 + lane));
  }
  float lo = 0.0f, hi = 0.0f;
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    const float2 c = __ldg(reinterpret_cast<const float2*>(w.vec + 2 * MLP_H) + 4 * n + t);  // w3
    float s0, s1, s2, s3;
    silu2(z2[n][0], z2[n][1], s0, s1);
    silu2(z2[n][2], z2[n][3], s2, s3);
    lo = fmaf(s0, c.x, lo);
    lo = fmaf(s1, c.y, lo);
    hi = fmaf(s2, c.x, hi);
    hi = fmaf(s3, c.y, hi);
  }
  lo += __shfl_xor_sync(0xffffffffu, lo, 1);
  lo += __shfl_xor_sync(0xffffffffu, lo, 2);
  hi += __shfl_xor_sync(0xffffffffu, hi, 1);
  hi += __shfl_xor_sync(0xffffffffu, hi, 2);
  const float b3 = __ldg(w.vec + 3 * MLP_H);
  y_lo = lo + b3;
  y_hi = hi + b3;
}

// Inference with one sample per lane: p[c] = BF16 pair (x_2c, x_2c+1) of
// this lane's scaled inputs (p[4] = x8, x9).  Returns this lane's output.
// Must be called by all 32 lanes.  The warp's 32 samples are two 16-row
// tiles, evaluated one after the other by mlp_tile_forward.
__device__ __forceinline__ float mlp_warp_eval(const MlpW& w, const uint32_t (&p)[5]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float out = 0.0f;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    uint32_t a0 = 0, a1 = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const uint32_t v0 = __shfl_sync(0xffffffffu, p[c], 16 * mt + g);
      const uint32_t v1 = __shfl_sync(0xffffffffu, p[c], 16 * mt + g + 8);
      if (t == c) {
        a0 = v0;
        a1 = v1;
      }
    }
    const uint32_t v0 = __shfl_sync(0xffffffffu, p[4], 16 * mt + g);
    const uint32_t v1 = __shfl_sync(0xffffffffu, p[4], 16 * mt + g + 8);
    const uint32_t a2 = t == 0 ? v0 : 0u, a3 = t == 0 ? v1 : 0u;
    float z1[8][4], z2[8][4], lo, hi;
    mlp_tile_forward(w, a0, a1, a2, a3, z1, z2, lo, hi);
    const int rr = lane & 15;
    const float vlo = __shfl_sync(0xffffffffu, lo, 4 * (rr & 7));
    const float vhi = __shfl_sync(0xffffffffu, hi, 4 * (rr & 7));
    if ((lane >> 4) == mt) out = rr < 8 ? vlo : vhi;
  }
  return out;
}

// The same evaluation with the warp's two 16-row tiles side by side: they
// share every weight fragment load, and layer 2 is taken one n-tile at a
// time with its SiLU and output products right after, so h2 is never held.
// Every value is formed in the order mlp_tile_forward uses (bias, then the
// k-steps of each MMA in order; the output sum over n-tiles, then over the
// row's four lanes, then b3): the results equal mlp_warp_eval's bit for
// bit.  Measured: it shortens a latency-bound step (the screened
// multicomponent propose) and slows a throughput-bound one (the fused
// lattice step), where mlp_warp_eval stays.
__device__ __forceinline__ float mlp_warp_eval_pair(const MlpW& w, const uint32_t (&p)[5]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t x[2][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    uint32_t a0 = 0, a1 = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const uint32_t v0 = __shfl_sync(0xffffffffu, p[c], 16 * mt + g);
      const uint32_t v1 = __shfl_sync(0xffffffffu, p[c], 16 * mt + g + 8);
      if (t == c) {
        a0 = v0;
        a1 = v1;
      }
    }
    const uint32_t v0 = __shfl_sync(0xffffffffu, p[4], 16 * mt + g);
    const uint32_t v1 = __shfl_sync(0xffffffffu, p[4], 16 * mt + g + 8);
    x[mt][0] = a0;
    x[mt][1] = a1;
    x[mt][2] = t == 0 ? v0 : 0u;
    x[mt][3] = t == 0 ? v1 : 0u;
  }
  // layer 1 and SiLU, two n-tiles (one layer-2 k-tile) at a time
  uint32_t h[2][4][4];
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    float z[2][2][4];
#pragma unroll
    for (int hn = 0; hn < 2; ++hn) {
      const int n = 2 * kk + hn;
      const float2 bb = __ldg(reinterpret_cast<const float2*>(w.vec) + 4 * n + t);  // b1[8n + 2t], +1
      const uint2 b = __ldg(w.w1f + n * 32 + lane);
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        z[hn][mt][0] = bb.x;
        z[hn][mt][1] = bb.y;
        z[hn][mt][2] = bb.x;
        z[hn][mt][3] = bb.y;
        mma_bf16(z[hn][mt], x[mt][0], x[mt][1], x[mt][2], x[mt][3], b);
      }
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      h[mt][kk][0] = silu_bf16x2(z[0][mt][0], z[0][mt][1]);
      h[mt][kk][1] = silu_bf16x2(z[0][mt][2], z[0][mt][3]);
      h[mt][kk][2] = silu_bf16x2(z[1][mt][0], z[1][mt][1]);
      h[mt][kk][3] = silu_bf16x2(z[1][mt][2], z[1][mt][3]);
    }
  }
  // layer 2, SiLU and the output products, one n-tile at a time
  float lo[2] = {0.0f, 0.0f}, hi[2] = {0.0f, 0.0f};
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    const float2 bb = __ldg(reinterpret_cast<const float2*>(w.vec + MLP_H) + 4 * n + t);  // b2
    float z[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      z[mt][0] = bb.x;
      z[mt][1] = bb.y;
      z[mt][2] = bb.x;
      z[mt][3] = bb.y;
    }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const uint2 b = __ldg(w.w2f + (n * 4 + kk) * 32 + lane);
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) mma_bf16(z[mt], h[mt][kk][0], h[mt][kk][1], h[mt][kk][2], h[mt][kk][3], b);
    }
    const float2 c = __ldg(reinterpret_cast<const float2*>(w.vec + 2 * MLP_H) + 4 * n + t);  // w3
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      float s0, s1, s2, s3;
      silu2(z[mt][0], z[mt][1], s0, s1);
      silu2(z[mt][2], z[mt][3], s2, s3);
      lo[mt] = fmaf(s0, c.x, lo[mt]);
      lo[mt] = fmaf(s1, c.y, lo[mt]);
      hi[mt] = fmaf(s2, c.x, hi[mt]);
      hi[mt] = fmaf(s3, c.y, hi[mt]);
    }
  }
  const float b3 = __ldg(w.vec + 3 * MLP_H);
  const int rr = lane & 15;
  float out = 0.0f;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    float l = lo[mt], u = hi[mt];
    l += __shfl_xor_sync(0xffffffffu, l, 1);
    l += __shfl_xor_sync(0xffffffffu, l, 2);
    u += __shfl_xor_sync(0xffffffffu, u, 1);
    u += __shfl_xor_sync(0xffffffffu, u, 2);
    const float vlo = __shfl_sync(0xffffffffu, l + b3, 4 * (rr & 7));
    const float vhi = __shfl_sync(0xffffffffu, u + b3, 4 * (rr & 7));
    if ((lane >> 4) == mt) out = rr < 8 ? vlo : vhi;
  }
  return out;
}

}  // namespace vcsgc
