// C ABI of the learned block-Jacobi correction's network (include/ba.h,
// "Learned block-Jacobi correction"): inference, the loss gradient and the
// training loop, all on the tensor-core kernels of ba_learn.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "ba.h"
#include "ba_internal.h"
#include "ba_learn.cuh"

using namespace ba;

namespace {

#define LCU(call)                                                                                  \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return set_error(e_ == cudaErrorMemoryAllocation ? BA_ERR_OOM : BA_ERR_CUDA, "%s failed: %s", \
                       #call, cudaGetErrorString(e_));                                             \
  } while (0)

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t set_attrs() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MLP_SMEM_FWD);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MLP_SMEM_TRAIN);
  done = e == cudaSuccess;
  return e;
}

int train_grid(int n) {
  int dev = 0, nsm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return std::max(1, std::min(nsm, (n + MLP_ROWS - 1) / MLP_ROWS));
}

// Scratch of one gradient evaluation: per-CTA partials, the reduced
// gradient and the loss.
struct GradScratch {
  float* part = nullptr;
  double* lpart = nullptr;
  double* grad = nullptr;
  double* loss = nullptr;
  int grid = 0;
  ~GradScratch() {
    cudaFree(part);
    cudaFree(lpart);
    cudaFree(grad);
    cudaFree(loss);
  }
  cudaError_t init(int g, int nloss) {
    grid = g;
    cudaError_t e = cudaMalloc(&part, (size_t)g * MLP_NPARAM * 4);
    if (e == cudaSuccess) e = cudaMalloc(&lpart, (size_t)g * 8);
    if (e == cudaSuccess) e = cudaMalloc(&grad, (size_t)MLP_NPARAM * 8);
    if (e == cudaSuccess) e = cudaMalloc(&loss, (size_t)std::max(1, nloss) * 8);
    return e;
  }
};

void enqueue_grad(const float* params, int n, int K, const float* X, const float* A, const float* Y, const float* Z,
                  const GradScratch& g, double* grad, double* loss, cudaStream_t s) {
  k_mlp_train<<<g.grid, MLP_THREADS, MLP_SMEM_TRAIN, s>>>(n, K, params, X, A, Y, Z, g.part, g.lpart);
  k_mlp_reduce<<<nblk(MLP_NPARAM, 256), 256, 0, s>>>(g.grid, n, g.part, g.lpart, grad, loss);
  count_launch(2);
}

}  // namespace

extern "C" {

ba_status ba_mlp_forward(const float* params, int n, const float* X, float* E_out, void* stream) {
  if (n < 0 || (n > 0 && (!params || !X || !E_out))) return set_error(BA_ERR_INVALID_ARG, "bad argument");
  if (n == 0) return BA_OK;
  LCU(set_attrs());
  k_mlp_forward<<<nblk(n, MLP_ROWS), MLP_THREADS, MLP_SMEM_FWD, (cudaStream_t)stream>>>(n, params, X, E_out);
  count_launch();
  LCU(cudaGetLastError());
  return BA_OK;
}

ba_status ba_mlp_loss_grad(const float* params, int n, int K, const float* X, const float* Ahat, const float* Yhat,
                           const float* Zhat, double* grad_out, double* loss_out, void* stream) {
  if (n < 1 || K < 1 || K > MLP_KMAX || !params || !X || !Ahat || !Yhat || !Zhat || !grad_out)
    return set_error(BA_ERR_INVALID_ARG, "need n >= 1, 1 <= K <= %d and non-NULL arrays", MLP_KMAX);
  LCU(set_attrs());
  cudaStream_t s = (cudaStream_t)stream;
  GradScratch g;
  LCU(g.init(train_grid(n), 1));
  enqueue_grad(params, n, K, X, Ahat, Yhat, Zhat, g, grad_out, g.loss, s);
  LCU(cudaGetLastError());
  double l = 0.0;
  LCU(cudaMemcpyAsync(&l, g.loss, 8, cudaMemcpyDeviceToHost, s));
  LCU(cudaStreamSynchronize(s));
  if (loss_out) *loss_out = l;
  return BA_OK;
}

ba_status ba_mlp_train(float* params, float* adam_m, float* adam_v, int n, int K, const float* X, const float* Ahat,
                       const float* Yhat, const float* Zhat, int epochs, int batch, double lr, double* loss_hist,
                       void* stream) {
  if (n < 1 || K < 1 || K > MLP_KMAX || epochs < 0 || batch < 1 || !(lr > 0) || !params || !adam_m || !adam_v ||
      !X || !Ahat || !Yhat || !Zhat)
    return set_error(BA_ERR_INVALID_ARG, "bad argument");
  LCU(set_attrs());
  cudaStream_t s = (cudaStream_t)stream;
  const int b = std::min(batch, n);
  const int nb = n / b;  // whole minibatches; a tail shorter than `batch` is left out
  GradScratch g;
  LCU(g.init(train_grid(b), std::max(1, epochs * nb)));
  int step = 0;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int i = 0; i < nb; ++i) {
      const long long r0 = (long long)i * b;
      enqueue_grad(params, b, K, X + r0 * MLP_FIN, Ahat + r0 * 45, Yhat + r0 * 9 * K, Zhat + r0 * 9 * K, g, g.grad,
                   g.loss + (long long)ep * nb + i, s);
      ++step;
      k_adam<<<nblk(MLP_NPARAM, 256), 256, 0, s>>>(params, adam_m, adam_v, g.grad, step, (float)lr, 0.9f, 0.999f,
                                                   1e-8f);
      count_launch();
    }
  }
  LCU(cudaGetLastError());
  if (loss_hist && epochs > 0) {
    std::vector<double> l((size_t)epochs * nb);
    LCU(cudaMemcpyAsync(l.data(), g.loss, l.size() * 8, cudaMemcpyDeviceToHost, s));
    LCU(cudaStreamSynchronize(s));
    for (int ep = 0; ep < epochs; ++ep) {
      double m = 0.0;
      for (int i = 0; i < nb; ++i) m += l[(size_t)ep * nb + i];
      loss_hist[ep] = m / nb;
    }
  } else {
    LCU(cudaStreamSynchronize(s));
  }
  return BA_OK;
}

}  // extern "C"
