// Measured arithmetic peak of the CUDA cores (ba_measure_fma_peak): the
// denominator of the ALU roofline that the FP64 path (and the FP32 recompute
// passes) are reported against.  A roofline needs the machine's own rate,
// not a datasheet figure: on this GPU the FP64 rate is a small fraction of
// the FP32 rate, and both follow the SM clock.
//
// The kernel runs NCHAIN independent fused-multiply-add chains per thread
// (enough independent work to cover the FMA latency at full occupancy), on
// a grid of 8 CTAs of 256 threads per SM.  The chains' values are combined
// and written only when they reach an impossible value, so the compiler
// keeps every FMA; the result is counted as 2 flops per FMA.
#include <cuda_runtime.h>

#include "ba.h"
#include "ba_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kCtasPerSm = 8;
constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_peak(int iters, T a, T b, T* __restrict__ sink) {
  T v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  if (s == (T)-1.2345e30) sink[blockIdx.x] = s;  // never true for the inputs below
}

template <typename T>
ba_status measure(int iters, double* tflops_out, cudaStream_t s) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return ba::set_error(BA_ERR_CUDA, "device query failed: %s", cudaGetErrorString(e));
  const int grid = nsm * kCtasPerSm;
  T* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.f, best = 0.f;
  e = cudaMalloc(&sink, sizeof(T) * grid);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // a = 1 - 2^-20, b = 2^-20: the chains stay near 1, finite and normal
  const T a = (T)(1.0 - 1.0 / 1048576.0), b = (T)(1.0 / 1048576.0);
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // first launch is a warm-up
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
      k_fma_peak<T><<<grid, kThreads, 0, s>>>(iters, a, b, sink);
      ba::count_launch();
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) return ba::set_error(BA_ERR_CUDA, "FMA peak measurement failed: %s", cudaGetErrorString(e));
  const double fmas = (double)grid * kThreads * kChains * (double)iters;
  *tflops_out = 2.0 * fmas / (best * 1e-3) / 1e12;
  return BA_OK;
}

}  // namespace

extern "C" ba_status ba_measure_fma_peak(int precision, double* tflops_out, void* stream) {
  if (!tflops_out || (precision != BA_PREC_F64 && precision != BA_PREC_F32))
    return ba::set_error(BA_ERR_INVALID_ARG, "precision must be BA_PREC_F64 or BA_PREC_F32 and tflops_out non-NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // about 10 ms per launch at the expected rates (FP32 has ~64x the FP64 rate)
  return precision == BA_PREC_F64 ? measure<double>(1 << 12, tflops_out, s) : measure<float>(1 << 18, tflops_out, s);
}
