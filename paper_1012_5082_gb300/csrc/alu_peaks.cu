// alu_peaks.cu -- standalone throughput probe of the arithmetic units the
// colour step and the MD force kernel lean on (not part of libvcsgc.so).
//
// Each kernel runs 8 SMs' worth of blocks per SM (blocks = 8 x SMs, 256
// threads) with independent dependency chains per thread, timed with CUDA
// events after one warm-up launch; the figures are per GPU.  Printed as one
// JSON object.  Build and run: python -m paper_1012_5082_gb300.alu_peaks
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

namespace {

template <typename T>
__global__ void k_fma(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) x[q] = (T)(threadIdx.x + q) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = x[q] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += x[q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_exp64(double* out, int iters) {
  double x = -(double)(threadIdx.x % 64) * 0.1, s = 0.0;
  for (int i = 0; i < iters; ++i) {
    s += exp(x);
    x -= 1e-7;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_exp32(float* out, int iters) {
  float x = -(float)(threadIdx.x % 64) * 0.1f, s = 0.0f;
  for (int i = 0; i < iters; ++i) {
    s += expf(x);
    x -= 1e-7f;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_tanh(float* out, int iters) {
  float x[4] = {threadIdx.x * 1e-4f, 0.1f, 0.2f, 0.3f};
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float y;
      asm volatile("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x[q]));
      x[q] = y + 1e-3f;
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x[0] + x[1] + x[2] + x[3];
}

__global__ void k_xor_add(unsigned* out, int iters, unsigned a) {
  unsigned x[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) x[q] = threadIdx.x * (2u * q + 1u);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = (x[q] ^ a) + x[(q + 1) & 7];
  }
  unsigned s = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += x[q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_popc(unsigned* out, int iters, unsigned a) {
  unsigned x0 = threadIdx.x, x1 = x0 * 3u, x2 = x0 * 5u, x3 = x0 * 7u, s = 0;
  for (int i = 0; i < iters; ++i) {
    s += __popc(x0 & a) + __popc(x1 & a) + __popc(x2 & a) + __popc(x3 & a);
    x0 += s;
    x1 ^= s;
    x2 += a;
    x3 ^= a;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s + x0 + x1 + x2 + x3;
}

__global__ void k_mulhilo(unsigned* out, int iters, unsigned a) {
  unsigned x[4] = {threadIdx.x, threadIdx.x * 3u, threadIdx.x * 5u, threadIdx.x * 7u};
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < 4; ++q) x[q] = __umulhi(x[q], a) ^ (x[q] * a);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x[0] + x[1] + x[2] + x[3];
}

// mma.sync m16n8k16 BF16 -> FP32: 4 independent accumulators per warp
__global__ void k_mma(float* out, int iters) {
  uint32_t a0 = 0x3f803f80u + threadIdx.x, a1 = a0 ^ 1u, a2 = a0 ^ 2u, a3 = a0 ^ 3u;
  uint32_t b0 = 0x3c003c00u, b1 = b0 ^ 5u;
  float d[4][4] = {};
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};\n"
          : "+f"(d[q][0]), "+f"(d[q][1]), "+f"(d[q][2]), "+f"(d[q][3])
          : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  float s = 0.0f;
#pragma unroll
  for (int q = 0; q < 4; ++q) s += d[q][0] + d[q][1] + d[q][2] + d[q][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

#define CHECK(x)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (x);                                                               \
    if (e_ != cudaSuccess) {                                                            \
      std::printf("{\"error\": \"%s: %s\"}\n", #x, cudaGetErrorString(e_));             \
      return 1;                                                                         \
    }                                                                                   \
  } while (0)

int main() {
  cudaDeviceProp p;
  CHECK(cudaGetDeviceProperties(&p, 0));
  const int blocks = p.multiProcessorCount * 8, threads = 256;
  const double nthr = (double)blocks * threads;
  void* buf = nullptr;
  CHECK(cudaMalloc(&buf, sizeof(double) * blocks * threads));
  double* d = static_cast<double*>(buf);
  float* f = static_cast<float*>(buf);
  unsigned* u = static_cast<unsigned*>(buf);
  cudaEvent_t e0, e1;
  CHECK(cudaEventCreate(&e0));
  CHECK(cudaEventCreate(&e1));
  auto timed = [&](auto launch) -> double {
    launch();  // warm-up
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms * 1e-3;
  };
  const int it64 = 4096, it32 = 65536, itx = 256, itf = 8192, itt = 8192, iti = 16384, itm = 4096;
  const double t_fma64 = timed([&] { k_fma<double><<<blocks, threads>>>(d, it64, 0.999999, 1e-7); });
  const double t_fma32 = timed([&] { k_fma<float><<<blocks, threads>>>(f, it32, 0.999999f, 1e-7f); });
  const double t_exp64 = timed([&] { k_exp64<<<blocks, threads>>>(d, itx); });
  const double t_exp32 = timed([&] { k_exp32<<<blocks, threads>>>(f, itf); });
  const double t_tanh = timed([&] { k_tanh<<<blocks, threads>>>(f, itt); });
  const double t_int = timed([&] { k_xor_add<<<blocks, threads>>>(u, iti, 0x9E3779B9u); });
  const double t_popc = timed([&] { k_popc<<<blocks, threads>>>(u, iti, 0x9E3779B9u); });
  const double t_mul = timed([&] { k_mulhilo<<<blocks, threads>>>(u, iti, 0xD2511F53u); });
  const double t_mma = timed([&] { k_mma<<<blocks, threads>>>(f, itm); });
  CHECK(cudaGetLastError());
  CHECK(cudaDeviceSynchronize());
  const double warps = nthr / 32.0;
  std::printf(
      "{\"gpu\": \"%s\", \"sms\": %d, \"fp64_fma_tflops\": %.3f, \"fp32_fma_tflops\": %.3f, "
      "\"fp64_exp_g_per_s\": %.2f, \"fp32_expf_g_per_s\": %.1f, \"tanh_approx_g_per_s\": %.1f, "
      "\"int32_xor_add_tops\": %.2f, \"popc_t_per_s\": %.2f, \"mulhi_lo_pairs_t_per_s\": %.2f, "
      "\"mma_sync_bf16_tflops\": %.1f}\n",
      p.name, p.multiProcessorCount, 2.0 * 8 * it64 * nthr / t_fma64 * 1e-12,
      2.0 * 8 * it32 * nthr / t_fma32 * 1e-12, itx * nthr / t_exp64 * 1e-9, itf * nthr / t_exp32 * 1e-9,
      4.0 * itt * nthr / t_tanh * 1e-9, 16.0 * iti * nthr / t_int * 1e-12, 4.0 * iti * nthr / t_popc * 1e-12,
      4.0 * iti * nthr / t_mul * 1e-12, 2.0 * 16 * 8 * 16 * 4.0 * itm * warps / t_mma * 1e-12);
  cudaFree(buf);
  return 0;
}
