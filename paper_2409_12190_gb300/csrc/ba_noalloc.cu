// ba_csr_build_noalloc: the stable key sort of ba_csr_build with its scratch
// space in a fixed device array instead of a cudaMalloc'd buffer.
//
// Who needs this: callers that must not allocate device memory once they are
// running -- a real-time loop that cannot afford cudaMalloc/cudaFree (both
// can synchronise the whole device and take unbounded time), a host process
// whose device memory is entirely owned by another allocator (a framework's
// caching pool, a fixed budget), or code certified to allocate only at
// start-up.  They pass their own input and output buffers; the sort's
// temporary keys, values and digit histograms live in the array below.
//
// Costs and limits:
//  - The array is a file-scope __device__ variable.  The library's module is
//    loaded on a device lazily, so the array is reserved there by the first
//    call of this entry point on that device (the address lookup below loads
//    the module); from then on the device holds BA_NOALLOC_MAX_KEYS * 16 bytes
//    (+ histograms) of it until the process exits.  Callers that may allocate
//    only at start-up make one warm-up call (n = 0 is enough) then, before any
//    stream capture.
//  - The device address is looked up on every call, with the caller's device
//    current, so it stays right after a cudaDeviceReset or under another
//    context (the module is loaded again and the array may move); after a
//    reset the next call reserves the array again, like a first call.
//  - All calls share the one array.  Two calls whose GPU work overlaps (on
//    different streams, or from different host threads) corrupt each other's
//    results; order them on one stream or synchronise between them.
//  - The array keeps whatever the previous call left in it.  The only state
//    that must start at zero, the out-of-range flag, is cleared on every call;
//    the histograms and temporary keys are fully rewritten before use.
#include <cuda_runtime.h>

#include "ba.h"
#include "ba_internal.h"

namespace {

constexpr long long kMaxKeys = BA_NOALLOC_MAX_KEYS;
constexpr long long kTile = 4096;  // keys per radix tile (the sort's tile size)
constexpr long long kMaxTiles = (kMaxKeys + kTile - 1) / kTile;
// temporary keys A/B and values A/B, then the [256][tiles] histogram, then the
// error flag (own 256-byte line)
constexpr long long kErrOffsetInts = 4 * kMaxKeys + 256 * kMaxTiles;
constexpr long long kScratchInts = kErrOffsetInts + 64;

__device__ __align__(256) int32_t g_noalloc_scratch[kScratchInts];

// Device address of g_noalloc_scratch in the current device's context.  In
// host code the symbol itself is only a host-side stand-in, so the real
// address is asked of the runtime, with the caller's device current, on every
// call.  Once the module is loaded that is a table lookup; no address is
// cached, because a device reset or a new context can move the array.
cudaError_t scratch_address(void** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = p;
  return cudaSuccess;
}

}  // namespace

extern "C" ba_status ba_csr_build_noalloc(const int32_t* keys, int n, int n_keys, int32_t* perm_out,
                                          int32_t* rowptr_out, void* stream) {
  if (n < 0 || n_keys < 1) return ba::set_error(BA_ERR_INVALID_ARG, "n must be >= 0 and n_keys >= 1");
  if (n > kMaxKeys)
    return ba::set_error(BA_ERR_INVALID_ARG, "ba_csr_build_noalloc: n = %d exceeds the fixed maximum of %lld keys",
                         n, kMaxKeys);
  if ((n > 0 && (!keys || !perm_out)) || !rowptr_out) return ba::set_error(BA_ERR_INVALID_ARG, "NULL argument");
  void* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess)
    return ba::set_error(BA_ERR_CUDA, "ba_csr_build_noalloc: scratch set-up failed: %s", cudaGetErrorString(e));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* d_err = static_cast<int*>(base) + kErrOffsetInts;
  e = cudaMemsetAsync(d_err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = ba::csr_build_async(keys, n, n_keys, perm_out, rowptr_out, base, d_err, s);
  int err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return ba::set_error(BA_ERR_CUDA, "csr build failed: %s", cudaGetErrorString(e));
  if (err) return ba::set_error(BA_ERR_INVALID_ARG, "key out of range [0, %d)", n_keys);
  return BA_OK;
}
