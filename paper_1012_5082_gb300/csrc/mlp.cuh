// mlp.cuh -- device pieces of the delayed-acceptance surrogate shared by the
// colour step (inference, one trial per lane) and the training kernels.
//
// Network: ten environment counts c (own B counts in shells 1-5, then the
// first-shell neighbours' summed B counts in shells 1-5) scaled to
// x = c / max_c, then z1 = W1 x + b1, h1 = SiLU(z1), z2 = W2 h1 + b2,
// h2 = SiLU(z2), g = w3 . h2 + b3 (g predicts E(site = B) - E(site = A)).
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
__device__ __forceinline__ float silu(float z) { return z * sigm(z); }
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
    h[kk][0] = bf16x2(silu(z1[2 * kk][0]), silu(z1[2 * kk][1]));
    h[kk][1] = bf16x2(silu(z1[2 * kk][2]), silu(z1[2 * kk][3]));
    h[kk][2] = bf16x2(silu(z1[2 * kk + 1][0]), silu(z1[2 * kk + 1][1]));
    h[kk][3] = bf16x2(silu(z1[2 * kk + 1][2]), silu(z1[2 * kk + 1][3]));
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
    lo = fmaf(silu(z2[n][0]), c.x, lo);
    lo = fmaf(silu(z2[n][1]), c.y, lo);
    hi = fmaf(silu(z2[n][2]), c.x, hi);
    hi = fmaf(silu(z2[n][3]), c.y, hi);
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
// Must be called by all 32 lanes.
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

}  // namespace vcsgc
