// alu_peaks.cu -- standalone probe of the arithmetic throughputs and the
// step latencies the colour step and the MD force kernel lean on (not part
// of libvcsgc.so).
//
// Throughputs: each kernel runs 8 blocks of 256 threads per SM with
// independent dependency chains per thread, timed with CUDA events after one
// warm-up launch; the figures are per GPU.
// Latencies: (1) a CUDA graph of 64 launches of a 504 x 128 kernel (the
// launch shape of one colour step of 80^3 x 8 replicas) that waits for its
// predecessor, reads one word and adds one atomic, with and without
// programmatic dependent launch: the floor of one step as its own kernel;
// (2) a cooperative kernel of 1-3 blocks per SM crossing 2000 grid-wide
// barriers (arrival counter plus a generation word, spin bounded by an
// iteration limit that sets an error flag): the floor of one step inside a
// persistent kernel.  Printed as one JSON object.
// Build and run: python -m paper_1012_5082_gb300.alu_peaks
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

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__global__ void k_step_floor(int* acc, const int* src, int j) {
  pdl_trigger();
  pdl_wait();
  __shared__ int sv;
  if (threadIdx.x == 0) sv = *(volatile const int*)(acc + ((j + 3) & 3));
  int v = __ldcg(src + (blockIdx.x * blockDim.x + threadIdx.x) % 4096);
  __syncthreads();
  v += sv;
  if (threadIdx.x == 0 && v == 123456789) acc[8] = v;
  if (threadIdx.x == 0) atomicAdd(acc + (j & 3), 1);
}

// grid barrier: bar[0] arrivals, bar[1] generation; a spin longer than
// max_spin iterations sets *err and every block returns at the next check
__global__ void k_barriers(unsigned* bar, int* err, int steps, long long max_spin) {
  volatile unsigned* gen = bar + 1;
  for (int s = 0; s < steps; ++s) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned g0 = *gen;
      __threadfence();
      if (atomicAdd(bar, 1u) == gridDim.x - 1) {
        bar[0] = 0;
        __threadfence();
        atomicAdd(const_cast<unsigned*>(gen), 1u);
      } else {
        long long n = 0;
        while (*gen == g0) {
          if (++n > max_spin) {
            atomicExch(err, 1);
            break;
          }
        }
      }
      __threadfence();
    }
    __syncthreads();
    if (*(volatile int*)err) return;
  }
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

  // (1) chain of step-shaped launches in a graph
  cudaStream_t st;
  CHECK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  int* acc = nullptr;
  CHECK(cudaMalloc(&acc, 16 * sizeof(int)));
  CHECK(cudaMemset(acc, 0, 16 * sizeof(int)));
  CHECK(cudaMemset(buf, 0, 4096 * sizeof(int)));
  const int G = 64, reps = 50;
  double chain_us[2];
  for (int pdl = 0; pdl < 2; ++pdl) {
    cudaGraph_t g;
    cudaGraphExec_t ge;
    CHECK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    for (int jj = 0; jj < G; ++jj) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(504);
      cfg.blockDim = dim3(128);
      cfg.stream = st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      at[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = at;
      cfg.numAttrs = (pdl && jj > 0) ? 1 : 0;
      cudaLaunchKernelEx(&cfg, k_step_floor, acc, (const int*)u, jj);
    }
    CHECK(cudaStreamEndCapture(st, &g));
    CHECK(cudaGraphInstantiate(&ge, g, 0));
    CHECK(cudaGraphLaunch(ge, st));
    CHECK(cudaStreamSynchronize(st));
    CHECK(cudaEventRecord(e0, st));
    for (int q = 0; q < reps; ++q) CHECK(cudaGraphLaunch(ge, st));
    CHECK(cudaEventRecord(e1, st));
    CHECK(cudaEventSynchronize(e1));
    float ms = 0.0f;
    CHECK(cudaEventElapsedTime(&ms, e0, e1));
    chain_us[pdl] = 1e3 * ms / (reps * G);
    cudaGraphExecDestroy(ge);
    cudaGraphDestroy(g);
  }

  // (2) grid-wide barriers of a cooperative kernel
  unsigned* bar = nullptr;
  int* err = nullptr;
  CHECK(cudaMalloc(&bar, 2 * sizeof(unsigned)));
  CHECK(cudaMalloc(&err, sizeof(int)));
  int per_sm = 0;
  CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_barriers, 128, 0));
  double bar_us[3] = {0.0, 0.0, 0.0};
  int bar_err = 0;
  for (int bps = 1; bps <= 3 && bps <= per_sm; ++bps) {
    CHECK(cudaMemset(bar, 0, 2 * sizeof(unsigned)));
    CHECK(cudaMemset(err, 0, sizeof(int)));
    int blocks_c = p.multiProcessorCount * bps, steps = 2000;
    long long max_spin = 2000000;
    void* args[] = {&bar, &err, &steps, &max_spin};
    CHECK(cudaEventRecord(e0, st));
    CHECK(cudaLaunchCooperativeKernel((void*)k_barriers, dim3(blocks_c), dim3(128), args, 0, st));
    CHECK(cudaEventRecord(e1, st));
    CHECK(cudaEventSynchronize(e1));
    float ms = 0.0f;
    CHECK(cudaEventElapsedTime(&ms, e0, e1));
    int herr = 0;
    CHECK(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
    bar_err |= herr;
    bar_us[bps - 1] = 1e3 * ms / steps;
  }
  std::printf(
      "{\"gpu\": \"%s\", \"sms\": %d, \"fp64_fma_tflops\": %.3f, \"fp32_fma_tflops\": %.3f, "
      "\"fp64_exp_g_per_s\": %.2f, \"fp32_expf_g_per_s\": %.1f, \"tanh_approx_g_per_s\": %.1f, "
      "\"int32_xor_add_tops\": %.2f, \"popc_t_per_s\": %.2f, \"mulhi_lo_pairs_t_per_s\": %.2f, "
      "\"mma_sync_bf16_tflops\": %.1f, \"step_chain_us\": %.3f, \"step_chain_pdl_us\": %.3f, "
      "\"grid_barrier_us\": [%.3f, %.3f, %.3f], \"grid_barrier_timeout\": %d}\n",
      p.name, p.multiProcessorCount, 2.0 * 8 * it64 * nthr / t_fma64 * 1e-12,
      2.0 * 8 * it32 * nthr / t_fma32 * 1e-12, itx * nthr / t_exp64 * 1e-9, itf * nthr / t_exp32 * 1e-9,
      4.0 * itt * nthr / t_tanh * 1e-9, 16.0 * iti * nthr / t_int * 1e-12, 4.0 * iti * nthr / t_popc * 1e-12,
      4.0 * iti * nthr / t_mul * 1e-12, 2.0 * 16 * 8 * 16 * 4.0 * itm * warps / t_mma * 1e-12, chain_us[0],
      chain_us[1], bar_us[0], bar_us[1], bar_us[2], bar_err);
  cudaFree(buf);
  cudaFree(acc);
  cudaFree(bar);
  cudaFree(err);
  cudaStreamDestroy(st);
  return 0;
}
