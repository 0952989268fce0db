// Stable device radix sort of observation keys and the CSR row pointers built
// from it: the "symbolic phase" of Sec. IV-B (which blocks multiply into which
// output block depends only on the index pattern; it is computed once per
// problem and cached).
//
// LSD radix sort, 8-bit digits, 4096-key tiles.  Each pass: per-tile digit
// histogram (shared-memory integer atomics: exact, order-free), one exclusive
// scan over the digit-major [256][tiles] table, and a scatter in which every
// key finds its rank among equal digits of its tile through warp match masks
// and per-warp counters -- so equal digits keep their input order and the
// whole sort is stable.  Values start as the key's index, so the output
// permutation orders ties by observation index: bit-exact with a counting
// sort.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ba_internal.h"

namespace ba {

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 16;                       // keys per lane per tile
constexpr int RS_PER_WARP = 32 * RS_ITEMS;         // 512
constexpr int RS_TILE = RS_WARPS * RS_PER_WARP;    // 4096
constexpr int RS_SCAN_THREADS = 1024;

__global__ void k_rs_check(const int32_t* __restrict__ keys, int n, int n_keys,
                           int* __restrict__ err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    int k = keys[i];
    if (k < 0 || k >= n_keys) atomicOr(err, 1);
  }
}

__global__ void k_rs_iota(int32_t* __restrict__ out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = i;
}

__global__ void __launch_bounds__(RS_THREADS)
k_rs_hist(const int32_t* __restrict__ keys, int n, int shift, int ntiles,
          int32_t* __restrict__ hist) {
  __shared__ int h[256];
  const int tile = blockIdx.x;
  for (int d = threadIdx.x; d < 256; d += RS_THREADS) h[d] = 0;
  __syncthreads();
  const long long base = (long long)tile * RS_TILE;
  for (int i = threadIdx.x; i < RS_TILE; i += RS_THREADS) {
    long long idx = base + i;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += RS_THREADS) hist[(long long)d * ntiles + tile] = h[d];
}

// Exclusive scan of len ints in place, one block.
__global__ void __launch_bounds__(RS_SCAN_THREADS)
k_rs_scan(int32_t* __restrict__ a, long long len) {
  __shared__ long long part[RS_SCAN_THREADS];
  const long long chunk = (len + RS_SCAN_THREADS - 1) / RS_SCAN_THREADS;
  const long long lo = threadIdx.x * chunk;
  const long long hi = lo + chunk < len ? lo + chunk : len;
  long long s = 0;
  for (long long i = lo; i < hi; ++i) s += a[i];
  part[threadIdx.x] = s;
  __syncthreads();
  // Hillis-Steele inclusive scan of the per-thread sums
  for (int off = 1; off < RS_SCAN_THREADS; off <<= 1) {
    long long v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  long long run = part[threadIdx.x] - s;
  for (long long i = lo; i < hi; ++i) {
    long long v = a[i];
    a[i] = (int32_t)run;
    run += v;
  }
}

__global__ void __launch_bounds__(RS_THREADS)
k_rs_scatter(const int32_t* __restrict__ keys_in, const int32_t* __restrict__ vals_in,
             int n, int shift, int ntiles, const int32_t* __restrict__ offs,
             int32_t* __restrict__ keys_out, int32_t* __restrict__ vals_out) {
  __shared__ int cnt[RS_WARPS][256];
  __shared__ int woff[RS_WARPS][256];
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int tile = blockIdx.x;
  for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&cnt[0][0])[i] = 0;
  __syncthreads();
  const long long base = (long long)tile * RS_TILE + (long long)warp * RS_PER_WARP;
  const unsigned lt = (1u << lane) - 1u;
  int local[RS_ITEMS], dig[RS_ITEMS], key[RS_ITEMS], val[RS_ITEMS];
#pragma unroll
  for (int it = 0; it < RS_ITEMS; ++it) {
    const long long idx = base + it * 32 + lane;
    const bool valid = idx < n;
    const int k = valid ? keys_in[idx] : 0;
    const int d = valid ? ((k >> shift) & 255) : 256;
    const int v = valid ? (vals_in ? vals_in[idx] : (int)idx) : 0;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lt);
    const int leader = __ffs(peers) - 1;
    const int before = d < 256 ? cnt[warp][d] : 0;
    __syncwarp();
    if (lane == leader && d < 256) cnt[warp][d] = before + __popc(peers);
    __syncwarp();
    local[it] = before + rank;
    dig[it] = d;
    key[it] = k;
    val[it] = v;
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += RS_THREADS) {
    int run = 0;
    for (int w = 0; w < RS_WARPS; ++w) {
      woff[w][d] = run;
      run += cnt[w][d];
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < RS_ITEMS; ++it) {
    const int d = dig[it];
    if (d < 256) {
      const long long pos = (long long)offs[(long long)d * ntiles + tile] + woff[warp][d] + local[it];
      keys_out[pos] = key[it];
      vals_out[pos] = val[it];
    }
  }
}

// rowptr[k] = first sorted position with key >= k; rowptr[n_keys] = n.
__global__ void k_rs_rowptr(const int32_t* __restrict__ sorted, int n, int n_keys,
                            int32_t* __restrict__ rowptr) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s > n) return;
  // keys are range-checked before this runs; the clamps only keep every
  // write inside rowptr[0..n_keys] whatever the input
  if (s == n) {
    const int lo = n > 0 ? min(max(sorted[n - 1], -1), n_keys - 1) : -1;
    for (int k = lo + 1; k <= n_keys; ++k) rowptr[k] = n;
    return;
  }
  const int k = min(max(sorted[s], -1), n_keys - 1);
  const int prev = s > 0 ? min(max(sorted[s - 1], -1), n_keys - 1) : -1;
  for (int kk = prev + 1; kk <= k; ++kk) rowptr[kk] = (int32_t)s;
}

int bits_for(int n_keys) {
  int b = 0;
  unsigned v = n_keys > 1 ? (unsigned)(n_keys - 1) : 0u;
  while (v) {
    ++b;
    v >>= 1;
  }
  return b;
}

}  // namespace

size_t csr_scratch_bytes(int n) {
  const long long ntiles = (n + RS_TILE - 1) / RS_TILE;
  size_t b = 4 * (size_t)n * sizeof(int32_t) + 256 * (size_t)(ntiles > 0 ? ntiles : 1) * sizeof(int32_t);
  return b + 256;
}

cudaError_t csr_build_async(const int32_t* keys, int n, int n_keys, int32_t* perm_out,
                            int32_t* rowptr_out, void* scratch, int* d_err, cudaStream_t s) {
  int32_t* kA = static_cast<int32_t*>(scratch);
  int32_t* kB = kA + n;
  int32_t* vA = kB + n;
  int32_t* vB = vA + n;
  int32_t* hist = vB + n;
  const int ntiles = (n + RS_TILE - 1) / RS_TILE;
  if (n > 0) {
    k_rs_check<<<(n + 255) / 256, 256, 0, s>>>(keys, n, n_keys, d_err);
    count_launch();
  }
  const int bits = bits_for(n_keys);
  const int passes = (bits + 7) / 8;
  const int32_t* sorted_keys = keys;
  if (n > 0 && passes == 0) {
    k_rs_iota<<<(n + 255) / 256, 256, 0, s>>>(perm_out, n);
    count_launch();
  }
  if (n > 0 && passes > 0) {
    const int32_t* kin = keys;
    const int32_t* vin = nullptr;
    for (int p = 0; p < passes; ++p) {
      int32_t* kout = (p & 1) ? kA : kB;
      int32_t* vout = (p == passes - 1) ? perm_out : ((p & 1) ? vA : vB);
      k_rs_hist<<<ntiles, RS_THREADS, 0, s>>>(kin, n, 8 * p, ntiles, hist);
      k_rs_scan<<<1, RS_SCAN_THREADS, 0, s>>>(hist, 256LL * ntiles);
      k_rs_scatter<<<ntiles, RS_THREADS, 0, s>>>(kin, vin, n, 8 * p, ntiles, hist, kout, vout);
      count_launch(3);
      kin = kout;
      vin = vout;
    }
    sorted_keys = kin;
  }
  k_rs_rowptr<<<(n + 1 + 255) / 256, 256, 0, s>>>(sorted_keys, n, n_keys, rowptr_out);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ba
