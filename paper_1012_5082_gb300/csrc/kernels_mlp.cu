// kernels_mlp.cu -- inference and training kernels of the delayed-acceptance
// surrogate (network and tensor-core form described in mlp.cuh).
//
// Training minimises the mean squared error of g against the exact energy
// change E(B) - E(A) with Adam.  One step = one launch of k_mlp_backward over
// a minibatch (drawn with replacement by Philox from the sample set, or the
// whole set in order) and one single-block launch of k_mlp_adam_pack that
// updates the FP32 master parameters and re-packs the BF16 fragments.  The
// step counter lives on the device, so a run of steps can be replayed as a
// CUDA graph.
//
// Backward pass of a 16-sample tile (one warp; operands BF16, sums FP32):
//   d3 = 2 (g - y) / B;  dw3 = sum_s d3 h2;  d2 = d3 w3 SiLU'(z2)
//   dW2 = d2^T h1 (MMA, samples as k);  dh1 = d2 W2 (MMA);  d1 = dh1 SiLU'(z1)
//   dW1 = d1^T x  (MMA);  biases: column sums of d1, d2, d3.
// Weight gradients are summed per block in shared memory and added to the
// global gradient once per block.
#include "common.cuh"
#include "kernels.h"
#include "mlp.cuh"

namespace vcsgc {

namespace {

constexpr uint32_t TAG_MLP_SAMPLE = 6u;
constexpr int TRAIN_WARPS = 4;

__device__ __forceinline__ uint32_t pack_raw(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// A(m, k) = M[(k0 + k) ld + r0 + m]   (transposed operand)
__device__ __forceinline__ void smem_at(uint32_t (&a)[4], const __nv_bfloat16* M, int ld, int r0, int k0) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const __nv_bfloat16* c0 = M + (k0 + 2 * t) * ld + r0 + g;
  a[0] = pack_raw(c0[0], c0[ld]);
  a[1] = pack_raw(c0[8], c0[ld + 8]);
  a[2] = pack_raw(c0[8 * ld], c0[9 * ld]);
  a[3] = pack_raw(c0[8 * ld + 8], c0[9 * ld + 8]);
}
// B(k, n) = M[(k0 + k) ld + n0 + n]
__device__ __forceinline__ uint2 smem_b_kn(const __nv_bfloat16* M, int ld, int n0, int k0) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const __nv_bfloat16* c0 = M + (k0 + 2 * t) * ld + n0 + g;
  return make_uint2(pack_raw(c0[0], c0[ld]), pack_raw(c0[8 * ld], c0[9 * ld]));
}

// sum over the 8 row groups g (lanes with equal t)
__device__ __forceinline__ float sum_rows(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 16);
  return v;
}

// A fragment of the scaled inputs of rows r0 (= tile row g) and r1 (= g + 8);
// rows with v0 / v1 false are zero
__device__ __forceinline__ void input_frag(const float* X, long long r0, long long r1, bool v0, bool v1,
                                           uint32_t& a0, uint32_t& a1, uint32_t& a2, uint32_t& a3) {
  const int t = threadIdx.x & 3;
  const int c = 2 * t;
  float x[4] = {0.0f, 0.0f, 0.0f, 0.0f}, y[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  if (v0) {
    x[0] = X[r0 * MLP_IN + c] * mlp_in_scale(c);
    x[1] = X[r0 * MLP_IN + c + 1] * mlp_in_scale(c + 1);
    if (t == 0) {
      x[2] = X[r0 * MLP_IN + 8] * mlp_in_scale(8);
      x[3] = X[r0 * MLP_IN + 9] * mlp_in_scale(9);
    }
  }
  if (v1) {
    y[0] = X[r1 * MLP_IN + c] * mlp_in_scale(c);
    y[1] = X[r1 * MLP_IN + c + 1] * mlp_in_scale(c + 1);
    if (t == 0) {
      y[2] = X[r1 * MLP_IN + 8] * mlp_in_scale(8);
      y[3] = X[r1 * MLP_IN + 9] * mlp_in_scale(9);
    }
  }
  a0 = bf16x2(x[0], x[1]);
  a1 = bf16x2(y[0], y[1]);
  a2 = bf16x2(x[2], x[3]);
  a3 = bf16x2(y[2], y[3]);
}

__global__ void __launch_bounds__(128) k_mlp_forward(MlpW w, const float* X, long long n, float* out) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const long long tiles = (n + 15) / 16;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long tile = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); tile < tiles;
       tile += nw) {
    const long long r0 = tile * 16 + g, r1 = r0 + 8;
    uint32_t a0, a1, a2, a3;
    input_frag(X, r0, r1, r0 < n, r1 < n, a0, a1, a2, a3);
    float z1[8][4], z2[8][4], lo, hi;
    mlp_tile_forward(w, a0, a1, a2, a3, z1, z2, lo, hi);
    if (t == 0) {
      if (r0 < n) out[r0] = lo;
      if (r1 < n) out[r1] = hi;
    }
  }
}

struct TrainTile {
  __nv_bfloat16 x[16 * 16];     // scaled inputs [sample][in]
  __nv_bfloat16 h[16 * MLP_H];  // h1, then d1 [sample][hidden]
  __nv_bfloat16 d2[16 * MLP_H]; // d2 [sample][hidden]
};

// Gradient of the mean squared error over B samples, added to grad[]; the
// minibatch row q is sample below(n, Philox(step, q)) when key_on, else q.
__global__ void __launch_bounds__(32 * TRAIN_WARPS)
    k_mlp_backward(MlpW w, const float* X, const float* Y, long long n, long long B, int key_on, uint2 key,
                   const long long* ctr, const long long* base, float* grad, double* loss_hist) {
  __shared__ float s_grad[MLP_NPARAM];
  __shared__ __align__(16) TrainTile s_tile[TRAIN_WARPS];
  __shared__ float s_loss;
  for (int q = threadIdx.x; q < MLP_NPARAM; q += blockDim.x) s_grad[q] = 0.0f;
  if (threadIdx.x == 0) s_loss = 0.0f;
  __syncthreads();
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  TrainTile& T = s_tile[wid];
  uint32_t* Tx = reinterpret_cast<uint32_t*>(T.x);
  uint32_t* Th = reinterpret_cast<uint32_t*>(T.h);
  uint32_t* Td = reinterpret_cast<uint32_t*>(T.d2);
  const long long step = ctr ? *ctr : 0;
  const long long li = ctr ? step - *base : 0;  // row of loss_hist
  const float inv_b = 1.0f / (float)B;
  const long long tiles = (B + 15) / 16;
  const long long nw = (long long)gridDim.x * TRAIN_WARPS;
  float loss_part = 0.0f;
  for (long long tile = (long long)blockIdx.x * TRAIN_WARPS + wid; tile < tiles; tile += nw) {
    const long long q0 = tile * 16 + g, q1 = q0 + 8;
    const bool v0 = q0 < B, v1 = q1 < B;
    long long r0 = q0, r1 = q1;
    if (key_on) {
      const uint32_t slo = (uint32_t)step, shi = (uint32_t)((unsigned long long)step >> 32);
      if (v0) {
        const uint4 u = philox4x32_10(make_uint4(slo, shi, (uint32_t)q0, TAG_MLP_SAMPLE), key);
        r0 = (long long)below64(u.x, u.y, (uint64_t)n);
      }
      if (v1) {
        const uint4 u = philox4x32_10(make_uint4(slo, shi, (uint32_t)q1, TAG_MLP_SAMPLE), key);
        r1 = (long long)below64(u.x, u.y, (uint64_t)n);
      }
    }
    uint32_t a0, a1, a2, a3;
    input_frag(X, r0, r1, v0, v1, a0, a1, a2, a3);
    // the input tile in shared memory (B operand of dW1): row-major [16][16]
    Tx[g * 8 + t] = a0;
    Tx[(g + 8) * 8 + t] = a1;
    Tx[g * 8 + t + 4] = a2;
    Tx[(g + 8) * 8 + t + 4] = a3;
    float z1[8][4], z2[8][4], ylo, yhi;
    mlp_tile_forward(w, a0, a1, a2, a3, z1, z2, ylo, yhi);
    // h1 tile (the same BF16 values the forward used as the layer-2 operand)
#pragma unroll
    for (int nn = 0; nn < 8; ++nn) {
      Th[(g * MLP_H + 8 * nn + 2 * t) >> 1] = silu_bf16x2(z1[nn][0], z1[nn][1]);
      Th[((g + 8) * MLP_H + 8 * nn + 2 * t) >> 1] = silu_bf16x2(z1[nn][2], z1[nn][3]);
    }
    const float e0 = v0 ? ylo - Y[r0] : 0.0f;
    const float e1 = v1 ? yhi - Y[r1] : 0.0f;
    if (t == 0) loss_part += e0 * e0 + e1 * e1;
    const float d3a = 2.0f * e0 * inv_b, d3b = 2.0f * e1 * inv_b;
    // output layer and d2 (FP32), d2 tile (BF16)
    float d2[8][4];
    const float* w3 = w.vec + 2 * MLP_H;
#pragma unroll
    for (int nn = 0; nn < 8; ++nn) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int col = 8 * nn + 2 * t + c;
        const float za = z2[nn][c], zb = z2[nn][2 + c];
        float ha, hb;
        silu2(za, zb, ha, hb);
        const float gw3 = sum_rows(d3a * ha + d3b * hb);
        if (g == 0) atomicAdd(&s_grad[MLP_OFF_W3 + col], gw3);
        const float wc = __ldg(w3 + col);
        d2[nn][c] = d3a * wc * dsilu(za);
        d2[nn][2 + c] = d3b * wc * dsilu(zb);
        const float gb2 = sum_rows(d2[nn][c] + d2[nn][2 + c]);
        if (g == 0) atomicAdd(&s_grad[MLP_OFF_B2 + col], gb2);
      }
      Td[(g * MLP_H + 8 * nn + 2 * t) >> 1] = bf16x2(d2[nn][0], d2[nn][1]);
      Td[((g + 8) * MLP_H + 8 * nn + 2 * t) >> 1] = bf16x2(d2[nn][2], d2[nn][3]);
    }
    const float gb3 = sum_rows(t == 0 ? d3a + d3b : 0.0f);
    if (lane == 0) atomicAdd(&s_grad[MLP_OFF_B3], gb3);
    __syncwarp();
    // dW2[o][i] = sum_s d2[s][o] h1[s][i]
#pragma unroll
    for (int mo = 0; mo < 4; ++mo) {
      uint32_t a[4];
      smem_at(a, T.d2, MLP_H, 16 * mo, 0);
#pragma unroll
      for (int ni = 0; ni < 8; ++ni) {
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        mma_bf16(acc, a[0], a[1], a[2], a[3], smem_b_kn(T.h, MLP_H, 8 * ni, 0));
        const int o0 = 16 * mo + g, i0 = 8 * ni + 2 * t;
        atomicAdd(&s_grad[MLP_OFF_W2 + o0 * MLP_H + i0], acc[0]);
        atomicAdd(&s_grad[MLP_OFF_W2 + o0 * MLP_H + i0 + 1], acc[1]);
        atomicAdd(&s_grad[MLP_OFF_W2 + (o0 + 8) * MLP_H + i0], acc[2]);
        atomicAdd(&s_grad[MLP_OFF_W2 + (o0 + 8) * MLP_H + i0 + 1], acc[3]);
      }
    }
    // dh1 = d2 W2 (A from the d2 registers), d1 = dh1 SiLU'(z1)
    uint32_t da[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      da[kk][0] = bf16x2(d2[2 * kk][0], d2[2 * kk][1]);
      da[kk][1] = bf16x2(d2[2 * kk][2], d2[2 * kk][3]);
      da[kk][2] = bf16x2(d2[2 * kk + 1][0], d2[2 * kk + 1][1]);
      da[kk][3] = bf16x2(d2[2 * kk + 1][2], d2[2 * kk + 1][3]);
    }
    __syncwarp();  // every lane has read h1 for dW2: the tile now takes d1
#pragma unroll
    for (int ni = 0; ni < 8; ++ni) {
      float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        mma_bf16(acc, da[kk][0], da[kk][1], da[kk][2], da[kk][3], __ldg(w.w2tf + (ni * 4 + kk) * 32 + lane));
      float d1[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) d1[c] = acc[c] * dsilu(z1[ni][c]);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float gb1 = sum_rows(d1[c] + d1[2 + c]);
        if (g == 0) atomicAdd(&s_grad[MLP_OFF_B1 + 8 * ni + 2 * t + c], gb1);
      }
      Th[(g * MLP_H + 8 * ni + 2 * t) >> 1] = bf16x2(d1[0], d1[1]);
      Th[((g + 8) * MLP_H + 8 * ni + 2 * t) >> 1] = bf16x2(d1[2], d1[3]);
    }
    __syncwarp();
    // dW1[o][i] = sum_s d1[s][o] x[s][i], i < 10
#pragma unroll
    for (int mo = 0; mo < 4; ++mo) {
      uint32_t a[4];
      smem_at(a, T.h, MLP_H, 16 * mo, 0);
#pragma unroll
      for (int ni = 0; ni < 2; ++ni) {
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        mma_bf16(acc, a[0], a[1], a[2], a[3], smem_b_kn(T.x, 16, 8 * ni, 0));
        const int o0 = 16 * mo + g, i0 = 8 * ni + 2 * t;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          if (i0 + c < MLP_IN) {
            atomicAdd(&s_grad[MLP_OFF_W1 + o0 * MLP_IN + i0 + c], acc[c]);
            atomicAdd(&s_grad[MLP_OFF_W1 + (o0 + 8) * MLP_IN + i0 + c], acc[2 + c]);
          }
        }
      }
    }
    __syncwarp();  // the tile is rewritten by the next iteration
  }
  loss_part += __shfl_xor_sync(0xffffffffu, loss_part, 4);
  loss_part += __shfl_xor_sync(0xffffffffu, loss_part, 8);
  loss_part += __shfl_xor_sync(0xffffffffu, loss_part, 16);
  if (lane == 0) atomicAdd(&s_loss, loss_part);
  __syncthreads();
  for (int q = threadIdx.x; q < MLP_NPARAM; q += blockDim.x)
    if (s_grad[q] != 0.0f) atomicAdd(&grad[q], s_grad[q]);
  if (threadIdx.x == 0 && loss_hist) atomicAdd(loss_hist + li, (double)s_loss * (double)inv_b);
}

// BF16 fragments and the FP32 vector of the parameters p (one block)
__device__ void pack_block(const float* p, uint2* w1f, uint2* w2f, uint2* w2tf, float* vec) {
  for (int q = threadIdx.x; q < MLP_W1F; q += blockDim.x) {
    const int n = q >> 5, lane = q & 31, g = lane >> 2, t = lane & 3;
    const int o = 8 * n + g;
    const int cols[4] = {2 * t, 2 * t + 1, 2 * t + 8, 2 * t + 9};
    float v[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] = cols[c] < MLP_IN ? p[MLP_OFF_W1 + o * MLP_IN + cols[c]] : 0.0f;
    w1f[q] = make_uint2(bf16x2(v[0], v[1]), bf16x2(v[2], v[3]));
  }
  const float* W2 = p + MLP_OFF_W2;
  for (int q = threadIdx.x; q < MLP_W2F; q += blockDim.x) {
    const int lane = q & 31, kk = (q >> 5) & 3, n = q >> 7, g = lane >> 2, t = lane & 3;
    const int o = 8 * n + g, k0 = 16 * kk + 2 * t;
    w2f[q] = make_uint2(bf16x2(W2[o * MLP_H + k0], W2[o * MLP_H + k0 + 1]),
                        bf16x2(W2[o * MLP_H + k0 + 8], W2[o * MLP_H + k0 + 9]));
    const int i = 8 * n + g;
    w2tf[q] = make_uint2(bf16x2(W2[k0 * MLP_H + i], W2[(k0 + 1) * MLP_H + i]),
                         bf16x2(W2[(k0 + 8) * MLP_H + i], W2[(k0 + 9) * MLP_H + i]));
  }
  for (int q = threadIdx.x; q < MLP_VEC; q += blockDim.x) {
    float v = 0.0f;
    if (q < MLP_H) v = p[MLP_OFF_B1 + q];
    else if (q < 2 * MLP_H) v = p[MLP_OFF_B2 + q - MLP_H];
    else if (q < 3 * MLP_H) v = p[MLP_OFF_W3 + q - 2 * MLP_H];
    else if (q == 3 * MLP_H) v = p[MLP_OFF_B3];
    vec[q] = v;
  }
}

__global__ void k_mlp_pack(const float* p, uint2* w1f, uint2* w2f, uint2* w2tf, float* vec) {
  pack_block(p, w1f, w2f, w2tf, vec);
}

// Adam (Kingma and Ba) on the FP32 parameters with step t = ctr[0] + 1 and
// a learning rate decaying from lr to lr / 100 by a half cosine over the
// `total` steps of the run that started at step ctr[1]; the gradient is
// cleared for the next step, the fragments re-packed and the counter
// advanced.
__global__ void __launch_bounds__(1024) k_mlp_adam_pack(float* p, float* m, float* v, float* grad, float lr,
                                                        long long total, long long* ctr, uint2* w1f, uint2* w2f,
                                                        uint2* w2tf, float* vec) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float t = (float)(ctr[0] + 1);
  if (total > 1) {
    const float f = (float)(ctr[0] - ctr[1]) / (float)(total - 1);
    lr *= 0.01f + 0.495f * (1.0f + cospif(fminf(f, 1.0f)));
  }
  const float c1 = 1.0f / (1.0f - powf(b1, t)), c2 = 1.0f / (1.0f - powf(b2, t));
  for (int q = threadIdx.x; q < MLP_NPARAM; q += blockDim.x) {
    const float gq = grad[q];
    const float mq = fmaf(b1, m[q], (1.0f - b1) * gq);
    const float vq = fmaf(b2, v[q], (1.0f - b2) * gq * gq);
    m[q] = mq;
    v[q] = vq;
    p[q] -= lr * (mq * c1) / (sqrtf(vq * c2) + eps);
    grad[q] = 0.0f;
  }
  __syncthreads();
  pack_block(p, w1f, w2f, w2tf, vec);
  __syncthreads();
  if (threadIdx.x == 0) *ctr += 1;
}

}  // namespace

MlpW mlp_view(const MlpBuf& b) { return MlpW{b.w1f, b.w2f, b.w2tf, b.vec}; }

void launch_mlp_pack(const float* p, const MlpBuf& b, cudaStream_t st) {
  k_mlp_pack<<<1, 1024, 0, st>>>(p, b.w1f, b.w2f, b.w2tf, b.vec);
}

void launch_mlp_forward(const MlpBuf& b, const float* X, long long n, float* out, cudaStream_t st) {
  if (n <= 0) return;
  const long long tiles = (n + 15) / 16;
  long long blocks = (tiles + 3) / 4;
  if (blocks > 8 * 152) blocks = 8 * 152;
  k_mlp_forward<<<(unsigned)blocks, 128, 0, st>>>(mlp_view(b), X, n, out);
}

void launch_mlp_backward(const MlpBuf& b, const float* X, const float* Y, long long n, long long B,
                         bool sample, uint2 key, const long long* ctr, const long long* base, float* grad,
                         double* loss_hist, cudaStream_t st) {
  if (B <= 0) return;
  const long long tiles = (B + 15) / 16;
  // each block ends with one global add per parameter: two tiles per warp,
  // at most one block per SM, the warps looping over the rest
  long long blocks = (tiles + 2 * TRAIN_WARPS - 1) / (2 * TRAIN_WARPS);
  if (blocks > 152) blocks = 152;
  k_mlp_backward<<<(unsigned)blocks, 32 * TRAIN_WARPS, 0, st>>>(mlp_view(b), X, Y, n, B, sample ? 1 : 0, key,
                                                                 ctr, base, grad, loss_hist);
}

void launch_mlp_adam_pack(float* p, float* m, float* v, float* grad, float lr, long long total, long long* ctr,
                          const MlpBuf& b, cudaStream_t st) {
  k_mlp_adam_pack<<<1, 1024, 0, st>>>(p, m, v, grad, lr, total, ctr, b.w1f, b.w2f, b.w2tf, b.vec);
}

}  // namespace vcsgc
