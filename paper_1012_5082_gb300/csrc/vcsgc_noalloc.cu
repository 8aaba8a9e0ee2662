// vcsgc_noalloc.cu -- neighbour-list build for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc at the point where they need a
// neighbour list: code that runs while another framework's caching allocator
// owns nearly all of the GPU's memory, code with a fixed memory budget set up
// once at start, or real-time loops that must not allocate.  They own their
// inputs (positions) and outputs (the list) and pass them in; the working
// space of the cell-list build lives in one file-scope device array instead.
//
// The array is a static __device__ symbol, so every GPU that loads this
// library holds it until the process exits.  Its address is obtained with
// cudaGetSymbolAddress once per device, with that device current, on the
// first call made on that device (that first call should come before any
// stream capture).  All calls share the array and it keeps the last call's
// contents; the call clears what has to start at zero.  Calls whose work
// overlaps on the GPU (e.g. on two streams at once) race on the array.
#include <mutex>

#include "../../include/vcsgc.h"
#include "common.cuh"
#include "kernels.h"

namespace {

using vcsgc::CellList;

constexpr long long NL_MAX_ATOMS = 262144;  // 2^18 positions
constexpr long long NL_MAX_CELLS = 65536;   // 2^16 binning cells

// layout (4-byte words): x32, y32, z32 [MAX_ATOMS each, float] |
//         cell_of[MAX_ATOMS] | sorted[MAX_ATOMS] | count[MAX_CELLS] |
//         start[MAX_CELLS + 1] | cursor[MAX_CELLS] | err (one word)
constexpr long long NL_SCRATCH_INTS = 5 * NL_MAX_ATOMS + 3 * NL_MAX_CELLS + 1 + 1;

static __device__ __align__(256) int g_nl_scratch[NL_SCRATCH_INTS];

constexpr int NL_MAX_DEVICES = 64;
std::mutex g_nl_mutex;
int* g_nl_ptr[NL_MAX_DEVICES] = {};

// errors are reported by code only (see include/vcsgc.h)
inline int nl_fail(int code, const char*) { return code; }
inline int nl_fail_cuda(const char*, cudaError_t) { return VCSGC_ERR_CUDA; }

}  // namespace

extern "C" int vcsgc_neighbour_list_noalloc(int64_t n, const double* d_x, const double* d_y,
                                            const double* d_z, const double box[3], double rl,
                                            int32_t K, int32_t* d_nbr, int32_t* d_cnt, void* stream) {
  if (n < 1 || !d_x || !d_y || !d_z || !box || !d_nbr || !d_cnt || K < 1 || !(rl > 0))
    return nl_fail(VCSGC_ERR_INVALID_ARG, "null pointer or non-positive size");
  if (n > NL_MAX_ATOMS) return nl_fail(VCSGC_ERR_INVALID_ARG, "more than 262144 positions");
  int nc[3];
  long long ncell = 1;
  for (int q = 0; q < 3; ++q) {
    if (!(box[q] > 2.0 * rl)) return nl_fail(VCSGC_ERR_INVALID_ARG, "box must exceed 2 rl");
    nc[q] = (int)(box[q] / rl);
    if (nc[q] < 3) return nl_fail(VCSGC_ERR_INVALID_ARG, "box must hold 3 cells of side rl");
    ncell *= nc[q];
  }
  if (ncell > NL_MAX_CELLS) return nl_fail(VCSGC_ERR_INVALID_ARG, "more than 65536 binning cells");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return nl_fail_cuda("cudaGetDevice", e);
  if (dev < 0 || dev >= NL_MAX_DEVICES) return nl_fail(VCSGC_ERR_INVALID_ARG, "device ordinal too large");
  int* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_nl_mutex);
    if (!g_nl_ptr[dev]) {
      e = cudaGetSymbolAddress((void**)&g_nl_ptr[dev], g_nl_scratch);
      if (e != cudaSuccess) {
        g_nl_ptr[dev] = nullptr;
        return nl_fail_cuda("cudaGetSymbolAddress", e);
      }
    }
    base = g_nl_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  CellList cl;
  cl.nc[0] = nc[0];
  cl.nc[1] = nc[1];
  cl.nc[2] = nc[2];
  cl.x32 = reinterpret_cast<float*>(base);
  cl.y32 = reinterpret_cast<float*>(base + NL_MAX_ATOMS);
  cl.z32 = reinterpret_cast<float*>(base + 2 * NL_MAX_ATOMS);
  cl.cell_of = base + 3 * NL_MAX_ATOMS;
  cl.sorted = base + 4 * NL_MAX_ATOMS;
  cl.cell_count = base + 5 * NL_MAX_ATOMS;
  cl.cell_start = cl.cell_count + NL_MAX_CELLS;
  cl.cell_cursor = cl.cell_start + NL_MAX_CELLS + 1;
  unsigned* err = reinterpret_cast<unsigned*>(cl.cell_cursor + NL_MAX_CELLS);
  // counts and cursors are cleared by the build itself; the error word here
  e = cudaMemsetAsync(err, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return nl_fail_cuda("cudaMemsetAsync", e);
  vcsgc::launch_cell_neighbours(n, d_x, d_y, d_z, box, rl, cl, K, d_nbr, d_cnt, err, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return nl_fail_cuda("launch", e);
  unsigned h_err = 0;
  e = cudaMemcpyAsync(&h_err, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return nl_fail_cuda("cudaMemcpyAsync", e);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return nl_fail_cuda("cudaStreamSynchronize", e);
  if (h_err & vcsgc::ERRF_OVERFLOW) return nl_fail(VCSGC_ERR_OVERFLOW, "a row had more than K neighbours (truncated)");
  return VCSGC_OK;
}
