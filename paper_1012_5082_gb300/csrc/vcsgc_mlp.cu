// vcsgc_mlp.cu -- C ABI of the delayed-acceptance surrogate network: an
// object holding the FP32 master parameters, Adam moments and the packed
// BF16 fragments on one GPU, with inference, a full-batch gradient and a
// training loop (minibatch Adam, replayed as a CUDA graph of 32 steps).
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/vcsgc.h"
#include "common.cuh"
#include "kernels.h"
#include "trace.h"

namespace {

using namespace vcsgc;

struct Mlp {
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::string err;
  float *p = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
  long long* ctr = nullptr;   // [0] = Adam step, [1] = step at the start of the current run
  double* loss = nullptr;
  long long loss_cap = 0;
  MlpBuf buf{};
  std::vector<void*> allocs;
};

#define MCK(call)                                                        \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) {                                             \
      m->err = std::string(#call) + ": " + cudaGetErrorString(e_);       \
      return VCSGC_ERR_CUDA;                                             \
    }                                                                    \
  } while (0)

template <typename T>
int malloc_n(Mlp* m, T** p, size_t n) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, sizeof(T) * (n ? n : 1));
  if (e != cudaSuccess) {
    cudaGetLastError();
    m->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    return VCSGC_ERR_NOMEM;
  }
  m->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return VCSGC_OK;
}

#define MTRY(x)                  \
  do {                           \
    int rc_ = (x);               \
    if (rc_ != VCSGC_OK) return rc_; \
  } while (0)

int upload(Mlp* m, const float* h) {
  MCK(cudaMemcpyAsync(m->p, h, sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice, m->st));
  MCK(cudaMemsetAsync(m->m, 0, sizeof(float) * MLP_NPARAM, m->st));
  MCK(cudaMemsetAsync(m->v, 0, sizeof(float) * MLP_NPARAM, m->st));
  MCK(cudaMemsetAsync(m->grad, 0, sizeof(float) * MLP_NPARAM, m->st));
  MCK(cudaMemsetAsync(m->ctr, 0, sizeof(long long) * 2, m->st));
  launch_mlp_pack(m->p, m->buf, m->st);
  MCK(cudaGetLastError());
  MCK(cudaStreamSynchronize(m->st));
  return VCSGC_OK;
}

void destroy(Mlp* m) {
  if (!m) return;
  if (m->st) cudaStreamSynchronize(m->st);
  for (void* q : m->allocs) cudaFree(q);
  if (m->own_stream && m->st) cudaStreamDestroy(m->st);
  delete m;
}

bool finite_params(const float* h) {
  for (int q = 0; q < MLP_NPARAM; ++q)
    if (!(h[q] == h[q]) || h[q] > 3.0e38f || h[q] < -3.0e38f) return false;
  return true;
}

}  // namespace

namespace vcsgc {
bool mlp_object_buffers(void* mlp, MlpBuf* out) {
  Mlp* m = static_cast<Mlp*>(mlp);
  if (!m) return false;
  *out = m->buf;
  return true;
}
cudaStream_t mlp_object_stream(void* mlp) { return static_cast<Mlp*>(mlp)->st; }
}  // namespace vcsgc

extern "C" {

int vcsgc_mlp_create(void** out, const float* params, void* stream) {
  if (!out || !params) return VCSGC_ERR_INVALID_ARG;
  *out = nullptr;
  if (!finite_params(params)) return VCSGC_ERR_NONFINITE;
  Mlp* m = new (std::nothrow) Mlp();
  if (!m) return VCSGC_ERR_NOMEM;
  m->st = static_cast<cudaStream_t>(stream);
  int rc = VCSGC_OK;
  if (!m->st) {
    // training is replayed as a graph: capture needs a stream of our own
    if (cudaStreamCreateWithFlags(&m->st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete m;
      return VCSGC_ERR_CUDA;
    }
    m->own_stream = true;
  }
  if (rc == VCSGC_OK) rc = malloc_n(m, &m->p, MLP_NPARAM);
  if (rc == VCSGC_OK) rc = malloc_n(m, &m->m, MLP_NPARAM);
  if (rc == VCSGC_OK) rc = malloc_n(m, &m->v, MLP_NPARAM);
  if (rc == VCSGC_OK) rc = malloc_n(m, &m->grad, MLP_NPARAM);
  if (rc == VCSGC_OK) rc = malloc_n(m, &m->ctr, 2);
  if (rc == VCSGC_OK) rc = malloc_n(m, &m->buf.w1f, MLP_W1F);
  if (rc == VCSGC_OK) rc = malloc_n(m, &m->buf.w2f, MLP_W2F);
  if (rc == VCSGC_OK) rc = malloc_n(m, &m->buf.w2tf, MLP_W2F);
  if (rc == VCSGC_OK) rc = malloc_n(m, &m->buf.vec, MLP_VEC);
  if (rc == VCSGC_OK) rc = upload(m, params);
  if (rc != VCSGC_OK) {
    destroy(m);
    return rc;
  }
  *out = m;
  return VCSGC_OK;
}

int vcsgc_mlp_set_params(void* mlp, const float* params) {
  Mlp* m = static_cast<Mlp*>(mlp);
  if (!m || !params) return VCSGC_ERR_INVALID_ARG;
  if (!finite_params(params)) return VCSGC_ERR_NONFINITE;
  return upload(m, params);
}

int vcsgc_mlp_get_params(void* mlp, float* params) {
  Mlp* m = static_cast<Mlp*>(mlp);
  if (!m || !params) return VCSGC_ERR_INVALID_ARG;
  MCK(cudaMemcpyAsync(params, m->p, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost, m->st));
  MCK(cudaStreamSynchronize(m->st));
  return VCSGC_OK;
}

int vcsgc_mlp_forward(void* mlp, const float* d_X, int64_t n, float* d_out) {
  VCSGC_TRACE("vcsgc_mlp_forward");
  Mlp* m = static_cast<Mlp*>(mlp);
  if (!m || n < 0 || (n > 0 && (!d_X || !d_out))) return VCSGC_ERR_INVALID_ARG;
  launch_mlp_forward(m->buf, d_X, n, d_out, m->st);
  MCK(cudaGetLastError());
  MCK(cudaStreamSynchronize(m->st));
  return VCSGC_OK;
}

int vcsgc_mlp_grad(void* mlp, const float* d_X, const float* d_Y, int64_t n, float* grad, double* loss) {
  VCSGC_TRACE("vcsgc_mlp_grad");
  Mlp* m = static_cast<Mlp*>(mlp);
  if (!m || !d_X || !d_Y || n < 1 || !grad || !loss) return VCSGC_ERR_INVALID_ARG;
  if (m->loss_cap < 1) {
    MTRY(malloc_n(m, &m->loss, 1));
    m->loss_cap = 1;
  }
  MCK(cudaMemsetAsync(m->grad, 0, sizeof(float) * MLP_NPARAM, m->st));
  MCK(cudaMemsetAsync(m->loss, 0, sizeof(double), m->st));
  launch_mlp_backward(m->buf, d_X, d_Y, n, n, false, make_uint2(0, 0), nullptr, nullptr, m->grad, m->loss, m->st);
  MCK(cudaGetLastError());
  MCK(cudaMemcpyAsync(grad, m->grad, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost, m->st));
  MCK(cudaMemcpyAsync(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->st));
  MCK(cudaMemsetAsync(m->grad, 0, sizeof(float) * MLP_NPARAM, m->st));
  MCK(cudaStreamSynchronize(m->st));
  return VCSGC_OK;
}

int vcsgc_mlp_train(void* mlp, const float* d_X, const float* d_Y, int64_t n, int64_t batch, int64_t steps,
                    double lr, uint64_t seed, double* loss_hist) {
  VCSGC_TRACE("vcsgc_mlp_train");
  Mlp* m = static_cast<Mlp*>(mlp);
  if (!m || !d_X || !d_Y || n < 1 || batch < 1 || steps < 0 || !(lr > 0.0) || n > (1LL << 40))
    return VCSGC_ERR_INVALID_ARG;
  if (steps == 0) return VCSGC_OK;
  if (m->loss_cap < steps) {
    MTRY(malloc_n(m, &m->loss, (size_t)steps));
    m->loss_cap = steps;
  }
  MCK(cudaMemsetAsync(m->loss, 0, sizeof(double) * steps, m->st));
  // base = the Adam step at the start of this run (loss rows count from it)
  MCK(cudaMemcpyAsync(m->ctr + 1, m->ctr, sizeof(long long), cudaMemcpyDeviceToDevice, m->st));
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  const float flr = (float)lr;
  auto one_step = [&]() {
    launch_mlp_backward(m->buf, d_X, d_Y, n, batch, true, key, m->ctr, m->ctr + 1, m->grad, m->loss, m->st);
    launch_mlp_adam_pack(m->p, m->m, m->v, m->grad, flr, (long long)steps, m->ctr, m->buf, m->st);
  };
  const int G = 32;
  long long left = steps;
  if (left >= G) {
    cudaGraph_t g;
    MCK(cudaStreamBeginCapture(m->st, cudaStreamCaptureModeThreadLocal));
    for (int q = 0; q < G; ++q) one_step();
    const cudaError_t e1 = cudaGetLastError();
    MCK(cudaStreamEndCapture(m->st, &g));
    if (e1 != cudaSuccess) {
      cudaGraphDestroy(g);
      m->err = std::string("capture: ") + cudaGetErrorString(e1);
      return VCSGC_ERR_CUDA;
    }
    cudaGraphExec_t ge = nullptr;
    const cudaError_t e2 = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) {
      m->err = std::string("graph: ") + cudaGetErrorString(e2);
      return VCSGC_ERR_CUDA;
    }
    cudaError_t e3 = cudaSuccess;
    while (left >= G && e3 == cudaSuccess) {
      e3 = cudaGraphLaunch(ge, m->st);
      left -= G;
    }
    const cudaError_t e4 = cudaStreamSynchronize(m->st);
    cudaGraphExecDestroy(ge);
    MCK(e3);
    MCK(e4);
  }
  for (; left > 0; --left) one_step();
  MCK(cudaGetLastError());
  if (loss_hist)
    MCK(cudaMemcpyAsync(loss_hist, m->loss, sizeof(double) * steps, cudaMemcpyDeviceToHost, m->st));
  MCK(cudaStreamSynchronize(m->st));
  return VCSGC_OK;
}

const char* vcsgc_mlp_last_error(void* mlp) {
  Mlp* m = static_cast<Mlp*>(mlp);
  return m ? m->err.c_str() : "null surrogate";
}

void vcsgc_mlp_free(void* mlp) { destroy(static_cast<Mlp*>(mlp)); }

}  // extern "C"
