// vcsgc_util.cu -- small entry points that expose device building blocks
// for checks against published values.
#include "../../include/vcsgc.h"
#include "common.cuh"
#include "trace.h"

namespace {

__global__ void k_philox_words(const uint4* ctr, const uint2* key, uint4* out, long long n) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) out[q] = vcsgc::philox4x32_10(ctr[q], key[q]);
}

}  // namespace

extern "C" int vcsgc_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n) {
  VCSGC_TRACE("vcsgc_philox");
  if (!ctr || !key || !out || n < 1 || n > (1LL << 20)) return VCSGC_ERR_INVALID_ARG;
  uint4* d_ctr = nullptr;
  uint2* d_key = nullptr;
  uint4* d_out = nullptr;
  int rc = VCSGC_OK;
  if (cudaMalloc(&d_ctr, sizeof(uint4) * n) != cudaSuccess || cudaMalloc(&d_key, sizeof(uint2) * n) != cudaSuccess ||
      cudaMalloc(&d_out, sizeof(uint4) * n) != cudaSuccess) {
    rc = VCSGC_ERR_NOMEM;
  } else if (cudaMemcpy(d_ctr, ctr, sizeof(uint4) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(d_key, key, sizeof(uint2) * n, cudaMemcpyHostToDevice) != cudaSuccess) {
    rc = VCSGC_ERR_CUDA;
  } else {
    k_philox_words<<<(unsigned)((n + 255) / 256), 256>>>(d_ctr, d_key, d_out, n);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(out, d_out, sizeof(uint4) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = VCSGC_ERR_CUDA;
  }
  cudaFree(d_ctr);
  cudaFree(d_key);
  cudaFree(d_out);
  return rc;
}
