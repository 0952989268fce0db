// Banded Cholesky of an SPD system A x = b and its two triangular solves in
// one cooperative launch (the paper's sparse direct solver, Sec. IV-C,
// "Sparse Direct Solver (Cholesky Factorization)").  It solves the damped
// pose-graph system H + D (Sec. IV-D), whose band is narrow, and the
// bundle-adjustment reduced camera system S (Eq. 2), whose band is the
// whole lower triangle.
//
// Storage.  In the factored order (for the pose graphs, reverse
// Cuthill-McKee when narrower) the matrix has half-bandwidth bw unknowns, so
// its lower triangle lies in the TB x TB tiles (I, J) with
// 0 <= I - J <= bwt = ceil(bw / TB).  Only those
// tiles are stored: tile (I, J) at T + (J (bwt + 1) + I - J) TB^2, row-major.
// The order is padded to nb TB unknowns with identity rows.  Cholesky keeps
// the fill inside the band, so L takes the same tiles.
//
// Tasks (a dependency graph; K0(I) = max(0, I - bwt) is the first column
// that reaches row I):
//   D_J     the diagonal chain: L_{J,J-1} = A_{J,J-1} L_{J-1,J-1}^{-T}, then
//           A_JJ -= L_{J,J-1} L_{J,J-1}^T and L_JJ = chol(A_JJ);
//   U       A_IJ -= L_IK L_JK^T for K in [Ka, Ka + cnt): the updates of a
//           tile, in ascending K (tile (J, J) leaves K = J - 1 to D_J);
//   T       L_IJ = A_IJ L_JJ^{-T} for I >= J + 2;
//   I_J     U_J = L_JJ^{-T} (the same solve with A = identity), so that the
//           triangular solves below are products, not serial substitutions;
//   F_J     y_J = U_J^T (b_J - sum_K L_JK y_K);
//   B_I     x_I = U_I (y_I - sum_K L_KI^T x_K).
// The chain D_0, D_1, ... is the critical path; one D_J is a triangular
// solve, a symmetric update and a factorisation of single tiles, while the U
// and T tasks of later columns run beside it.  The host orders the tasks by
// a list-scheduling simulation (a topological order) and splits them into two
// pools: the near-diagonal tasks that feed the chain, run by a few blocks of
// their own, and the bulk, run by the rest; each pool's blocks take its tasks
// in order from an atomic ticket.  A task waits only on tasks earlier in the
// simulated order.  The earliest unfinished task of that order has every
// predecessor done; if no block holds it, every block of its pool holds an
// earlier task of the same pool, which is impossible.  So the schedule cannot
// deadlock; every wait is bounded all the same (2^25 polls, about a second or
// more), and one that runs out sets ctr[3], after which every block stops.
//
// Each entry of L is a fixed-order sum (K ascending, then the tile's own
// columns), so the result does not depend on the schedule.
#pragma once

#include <cuda/atomic>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ba_band_sched.h"
#include "ba_dense.cuh"

namespace ba {

constexpr int BAND_TB = DB;        // tile size (32)
constexpr int BAND_THREADS = 256;  // threads per block
constexpr int BAND_TRI = BAND_TB * (BAND_TB + 1) / 2;  // entries of a tile's lower triangle

// The launch's arguments; the tasks are ba_band_sched.h's BandTask records,
// read as int4.
struct BandArgs {
  int nb;             // block rows of the padded order (nb * TB >= n)
  int bwt;            // half-bandwidth in tiles
  int n;              // unknowns
  int ntask;          // tasks
  int ncrit;          // the near-diagonal pool's tasks (the first ncrit of the list)
  int ncta_crit;      // blocks 0 .. ncta_crit - 1 run that pool
  const int4* task;   // [ntask] in ticket order, per pool
  double* T;          // band tiles, L on return
  double* rsd;        // [nb TB] 1 / L_cc of every diagonal entry
  double* Ui;         // [nb TB TB] U_J = L_JJ^{-T}, row-major (upper triangular)
  const double* rhs;  // [n] b
  double* y;          // [nb TB] y, then x
  double* sol;        // [n] x
  int* tflag;         // [nb (bwt + 1)] tile final (L)
  int* tprog;         // [nb (bwt + 1)] updates applied to the tile
  int* ctr;           // [0] bulk ticket, [1] forward blocks done, [2] backward blocks done, [3] a wait ran out,
                      // [4] near-diagonal ticket
  int* fail;          // a pivot not positive or not finite
  int* iflag;         // [nb] U_J final
};

__device__ __forceinline__ long long band_index(const BandArgs& a, int I, int J) {
  return (long long)J * (a.bwt + 1) + (I - J);
}

__device__ __forceinline__ double* band_tile(const BandArgs& a, int I, int J) {
  return a.T + band_index(a, I, J) * (BAND_TB * BAND_TB);
}

__device__ __forceinline__ int* band_flag(const BandArgs& a, int I, int J) { return a.tflag + band_index(a, I, J); }

__device__ __forceinline__ int* band_prog(const BandArgs& a, int I, int J) { return a.tprog + band_index(a, I, J); }

__device__ __forceinline__ int band_k0(const BandArgs& a, int I) { return max(0, I - a.bwt); }

// Thread-0 wait until *flag >= v (acquire).  False when the wait ran out or
// another one did (ctr[3]).
static __device__ __noinline__ bool band_wait(int* flag, int v, int* err) {
  cuda::atomic_ref<int, cuda::thread_scope_device> f(*flag), e(*err);
  unsigned int spins = 0;
  while (f.load(cuda::memory_order_acquire) < v) {
    if (e.load(cuda::memory_order_relaxed) || ++spins > (1u << 25)) {
      e.store(1, cuda::memory_order_relaxed);
      return false;
    }
    if (spins > 64) __nanosleep(64);
  }
  return true;
}

// Publish v after the block's writes (called by every thread).
__device__ __forceinline__ void band_publish(int* flag, int v) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    cuda::atomic_ref<int, cuda::thread_scope_device> f(*flag);
    f.store(v, cuda::memory_order_release);
  }
}

typedef double BandTile[BAND_TB][BAND_TB + 1];

// Stage a tile (row-major, TB x TB) into shared memory, through L2.
__device__ __forceinline__ void band_stage(BandTile& s, const double* __restrict__ g) {
  for (int e = threadIdx.x; e < BAND_TB * BAND_TB; e += BAND_THREADS) s[e / BAND_TB][e % BAND_TB] = __ldcg(g + e);
}

__device__ __forceinline__ void band_store(double* __restrict__ g, const BandTile& t) {
  for (int e = threadIdx.x; e < BAND_TB * BAND_TB; e += BAND_THREADS) g[e] = t[e / BAND_TB][e % BAND_TB];
}

struct BandSmem {
  BandTile A, B, C;
  double rs[BAND_TB];
  double d[BAND_TB];
  double red[BAND_THREADS / 32][BAND_TB];
  uint16_t tri[BAND_TRI];  // (r << 8) | c of the row-major lower triangle
  int task;
  int bad;
};

// X L^T = A in place (s.A = A on entry, X on return), L = the staged tile
// s.B with 1 / L_cc in s.rs: column by column, x_rc = a_rc / L_cc, then
// a_rc' -= x_rc L_c'c for c' > c (L's column c prescaled by 1 / L_cc; the
// prescaling overwrites s.B).
static __device__ void band_trsm(BandSmem& s) {
  constexpr int TB = BAND_TB;
  const int tid = threadIdx.x, lane = tid % 32, wp = tid / 32;
  for (int e = tid; e < TB * TB; e += BAND_THREADS) {
    const int rr = e / TB, cc = e % TB;
    if (rr > cc) s.B[rr][cc] *= s.rs[cc];
  }
  __syncthreads();
  for (int c = 0; c < TB - 1; ++c) {
    const double x = s.A[lane][c];
    for (int cp = c + 1 + wp; cp < TB; cp += BAND_THREADS / 32) s.A[lane][cp] = fma(-x, s.B[cp][c], s.A[lane][cp]);
    __syncthreads();
  }
  for (int e = tid; e < TB * TB; e += BAND_THREADS) s.A[e / TB][e % TB] *= s.rs[e % TB];
  __syncthreads();
}

// Factor the diagonal tile in s.C (lower triangle) into L, in place, with
// 1 / L_cc in s.rs: right-looking, one barrier per column; the scaling of
// column c is deferred (a_rc' -= a_rc a_c'c / d_c).  Lane 0 of warp 0
// updates each next pivot and takes its reciprocal square root, the serial
// chain of the factorisation; the other entries of the trailing triangle go
// to warps 1-3 and 5-7, so that the chain's FP64 instructions do not queue
// behind theirs (warps w and w + 4 share a scheduler).  A pivot that is not
// positive or not finite is replaced by 1 and counted in s.bad.
static __device__ void band_potrf(BandSmem& s) {
  constexpr int TB = BAND_TB, NU = BAND_THREADS - 64;  // updating threads
  const int tid = threadIdx.x, wp = tid / 32;
  const bool pivot = tid == 0;
  const bool upd = wp % 4 != 0;
  const int u = (wp < 4 ? wp - 1 : wp - 2) * 32 + tid % 32;  // 0 .. NU - 1 for the updating warps
  if (pivot) {
    const double d0 = s.C[0][0];
    const bool ok = d0 > 0.0 && isfinite(d0);
    s.d[0] = ok ? d0 : 1.0;
    s.rs[0] = ok ? rsqrt(d0) : 1.0;
    s.bad = ok ? 0 : 1;
  }
  __syncthreads();
  for (int c = 0; c < TB - 1; ++c) {
    const int m = TB - 1 - c, ne = m * (m + 1) / 2;
    const double inv = s.rs[c] * s.rs[c];
    if (pivot) {  // (c + 1, c + 1): the next pivot
      const double a = s.C[c + 1][c];
      const double v = fma(-(a * inv), a, s.C[c + 1][c + 1]);
      s.C[c + 1][c + 1] = v;
      const bool ok = v > 0.0 && isfinite(v);
      s.d[c + 1] = ok ? v : 1.0;
      s.rs[c + 1] = ok ? rsqrt(v) : 1.0;
      if (!ok) s.bad = 1;
    } else if (upd) {
      for (int e = 1 + u; e < ne; e += NU) {
        const int rr = c + 1 + (s.tri[e] >> 8), cc = c + 1 + (s.tri[e] & 0xff);
        s.C[rr][cc] = fma(-(s.C[rr][c] * inv), s.C[cc][c], s.C[rr][cc]);
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < TB * TB; e += BAND_THREADS) {
    const int rr = e / TB, cc = e % TB;
    s.C[rr][cc] = rr > cc ? s.C[rr][cc] * s.rs[cc] : (rr == cc ? s.d[cc] * s.rs[cc] : 0.0);
  }
  __syncthreads();
}

// D_J: the subdiagonal tile's solve, the last update of the diagonal tile
// and its factorisation.
static __device__ bool band_task_D(const BandArgs& a, BandSmem& s, int J) {
  constexpr int TB = BAND_TB;
  const int tid = threadIdx.x;
  if (J >= 1 && a.bwt >= 1) {
    // tiles (J, J - 1) and (J, J) hold every update before K = J - 1
    // (the two tiles of row J usually finish first: stage them while
    // L_{J-1,J-1} is still being factored)
    const int nupd = (J - 1) - band_k0(a, J);
    int w = 1;
    if (tid == 0)
      w = band_wait(band_prog(a, J, J - 1), nupd, a.ctr + 3) && band_wait(band_prog(a, J, J), nupd, a.ctr + 3);
    if (!__syncthreads_and(w)) return false;
    band_stage(s.A, band_tile(a, J, J - 1));
    band_stage(s.C, band_tile(a, J, J));
    w = 1;
    if (tid == 0) w = band_wait(band_flag(a, J - 1, J - 1), 1, a.ctr + 3);
    if (!__syncthreads_and(w)) return false;
    band_stage(s.B, band_tile(a, J - 1, J - 1));
    if (tid < TB) s.rs[tid] = __ldcg(a.rsd + (long long)(J - 1) * TB + tid);
    __syncthreads();
    band_trsm(s);  // s.A = L_{J,J-1}
    band_store(band_tile(a, J, J - 1), s.A);
    band_publish(band_flag(a, J, J - 1), 1);
    // A_JJ -= L_{J,J-1} L_{J,J-1}^T on the lower triangle
    for (int e = tid; e < BAND_TRI; e += BAND_THREADS) {
      const int r = s.tri[e] >> 8, c = s.tri[e] & 0xff;
      double v = s.C[r][c];
#pragma unroll 8
      for (int k = 0; k < TB; ++k) v = fma(-s.A[r][k], s.A[c][k], v);
      s.C[r][c] = v;
    }
    __syncthreads();
  } else {
    band_stage(s.C, band_tile(a, J, J));
    __syncthreads();
  }
  band_potrf(s);  // s.C = L_JJ
  band_store(band_tile(a, J, J), s.C);
  if (tid < TB) a.rsd[(long long)J * TB + tid] = s.rs[tid];
  if (tid == 0 && s.bad) atomicExch(a.fail, 1);
  band_publish(band_flag(a, J, J), 1);
  return true;
}

// U: A_IJ -= L_IK L_JK^T for K = Ka .. Ka + cnt - 1, after the tile's
// earlier updates.
static __device__ bool band_task_U(const BandArgs& a, BandSmem& s, int I, int J, int Ka, int cnt) {
  constexpr int TB = BAND_TB, E = TB * TB / BAND_THREADS, RS = BAND_THREADS / TB;
  const int tid = threadIdx.x, col = tid % TB, row0 = tid / TB;
  const int k0 = band_k0(a, I);
  int w = 1;
  if (tid == 0) w = band_wait(band_prog(a, I, J), Ka - k0, a.ctr + 3);
  if (!__syncthreads_and(w)) return false;
  double* Tij = band_tile(a, I, J);
  double acc[E];
#pragma unroll
  for (int m = 0; m < E; ++m) acc[m] = __ldcg(Tij + (row0 + m * RS) * TB + col);
  for (int K = Ka; K < Ka + cnt; ++K) {
    w = 1;
    if (tid == 0) w = band_wait(band_flag(a, I, K), 1, a.ctr + 3) && band_wait(band_flag(a, J, K), 1, a.ctr + 3);
    if (!__syncthreads_and(w)) return false;
    band_stage(s.A, band_tile(a, I, K));
    if (I != J) band_stage(s.B, band_tile(a, J, K));
    __syncthreads();
    const BandTile& LJ = (I != J) ? s.B : s.A;
#pragma unroll 8
    for (int k = 0; k < TB; ++k) {
      const double b = LJ[col][k];
#pragma unroll
      for (int m = 0; m < E; ++m) acc[m] = fma(-s.A[row0 + m * RS][k], b, acc[m]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int m = 0; m < E; ++m) Tij[(row0 + m * RS) * TB + col] = acc[m];
  band_publish(band_prog(a, I, J), Ka + cnt - k0);
  return true;
}

// T: L_IJ = A_IJ L_JJ^{-T} (I >= J + 2) after the tile's updates.
static __device__ bool band_task_T(const BandArgs& a, BandSmem& s, int I, int J) {
  constexpr int TB = BAND_TB;
  const int tid = threadIdx.x;
  int w = 1;
  if (tid == 0)
    w = band_wait(band_flag(a, J, J), 1, a.ctr + 3) && band_wait(band_prog(a, I, J), J - band_k0(a, I), a.ctr + 3);
  if (!__syncthreads_and(w)) return false;
  band_stage(s.A, band_tile(a, I, J));
  band_stage(s.B, band_tile(a, J, J));
  if (tid < TB) s.rs[tid] = __ldcg(a.rsd + (long long)J * TB + tid);
  __syncthreads();
  band_trsm(s);
  band_store(band_tile(a, I, J), s.A);
  band_publish(band_flag(a, I, J), 1);
  return true;
}

// I_J: U_J = L_JJ^{-T}, the solution of X L_JJ^T = identity.
static __device__ bool band_task_I(const BandArgs& a, BandSmem& s, int J) {
  constexpr int TB = BAND_TB;
  const int tid = threadIdx.x;
  int w = 1;
  if (tid == 0) w = band_wait(band_flag(a, J, J), 1, a.ctr + 3);
  if (!__syncthreads_and(w)) return false;
  band_stage(s.B, band_tile(a, J, J));
  if (tid < TB) s.rs[tid] = __ldcg(a.rsd + (long long)J * TB + tid);
  for (int e = tid; e < TB * TB; e += BAND_THREADS) s.A[e / TB][e % TB] = (e / TB == e % TB) ? 1.0 : 0.0;
  __syncthreads();
  band_trsm(s);
  band_store(a.Ui + (long long)J * TB * TB, s.A);
  band_publish(a.iflag + J, 1);
  return true;
}

__device__ __forceinline__ int band_load(int* p) {
  cuda::atomic_ref<int, cuda::thread_scope_device> f(*p);
  return f.load(cuda::memory_order_acquire);
}

// Thread 0: wait until the counter *p reaches v; *known caches the last value
// read, so a satisfied wait costs no load.
__device__ __forceinline__ bool band_wait_count(int* p, int v, int* known, int* err) {
  if (*known >= v) return true;
  *known = band_load(p);
  if (*known >= v) return true;
  if (!band_wait(p, v, err)) return false;
  *known = v;
  return true;
}

// Forward block F_J: y_J = L_JJ^{-1} (b_J - sum_{K < J} L_JK y_K).
static __device__ bool band_forward_task(const BandArgs& a, BandSmem& s, int J) {
  constexpr int TB = BAND_TB;
  const int tid = threadIdx.x, r = tid / 8, q = tid % 8;  // row r, columns 4q .. 4q + 3
  int known = 0;                                         // forward blocks known done (thread 0)
  double part = 0.0;
  for (int K = max(0, J - a.bwt); K < J; ++K) {
    int w = 1;
    if (tid == 0)
      w = band_wait(band_flag(a, J, K), 1, a.ctr + 3) && band_wait_count(a.ctr + 1, K + 1, &known, a.ctr + 3);
    if (!__syncthreads_and(w)) return false;
    const double* L = band_tile(a, J, K) + r * TB + 4 * q;
    const double* yk = a.y + (long long)K * TB + 4 * q;
#pragma unroll
    for (int c = 0; c < 4; ++c) part = fma(__ldcg(L + c), __ldcg(yk + c), part);
  }
  part += __shfl_xor_sync(0xffffffffu, part, 4);
  part += __shfl_xor_sync(0xffffffffu, part, 2);
  part += __shfl_xor_sync(0xffffffffu, part, 1);
  const long long row = (long long)J * TB + r;
  if (q == 0) s.d[r] = (row < a.n ? a.rhs[row] : 0.0) - part;
  int w = 1;
  if (tid == 0) w = band_wait(a.iflag + J, 1, a.ctr + 3);
  if (!__syncthreads_and(w)) return false;
  {
    // y = U_J^T v: lane r, rows c = wp, wp + 8, ... of U_J, summed over the
    // warps in order
    const int lane = tid % 32, wp = tid / 32;
    const double* U = a.Ui + (long long)J * TB * TB;
    double p = 0.0;
#pragma unroll
    for (int m = 0; m < TB / (BAND_THREADS / 32); ++m) {
      const int c = wp + m * (BAND_THREADS / 32);
      p = fma(__ldcg(U + c * TB + lane), s.d[c], p);
    }
    s.red[wp][lane] = p;
    __syncthreads();
    if (tid < 32) {
      double v = 0.0;
#pragma unroll
      for (int k = 0; k < BAND_THREADS / 32; ++k) v += s.red[k][lane];
      a.y[(long long)J * TB + lane] = v;
    }
  }
  // blocks are published in order (F_{J-1} first)
  w = 1;
  if (tid == 0) w = band_wait_count(a.ctr + 1, J, &known, a.ctr + 3);
  if (!__syncthreads_and(w)) return false;
  band_publish(a.ctr + 1, J + 1);
  return true;
}

// Backward block B_I: x_I = L_II^{-T} (y_I - sum_{K > I} L_KI^T x_K); x
// overwrites y.
static __device__ bool band_backward_task(const BandArgs& a, BandSmem& s, int I) {
  constexpr int TB = BAND_TB;
  const int tid = threadIdx.x, lane = tid % 32, wp = tid / 32;  // x row lane; L rows wp, wp + 8, ...
  int known = 0;                                                // backward blocks known done (thread 0)
  int w = 1;
  if (tid == 0) w = band_wait(a.ctr + 1, a.nb, a.ctr + 3);  // every tile and y final
  if (!__syncthreads_and(w)) return false;
  double part = 0.0;
  for (int K = min(a.nb - 1, I + a.bwt); K > I; --K) {
    w = 1;
    if (tid == 0) w = band_wait_count(a.ctr + 2, a.nb - K, &known, a.ctr + 3);
    if (!__syncthreads_and(w)) return false;
    const double* L = band_tile(a, K, I);
    const double* xk = a.y + (long long)K * TB;
#pragma unroll
    for (int m = 0; m < TB / (BAND_THREADS / 32); ++m) {
      const int c = wp + m * (BAND_THREADS / 32);
      part = fma(__ldcg(L + c * TB + lane), __ldcg(xk + c), part);
    }
  }
  s.red[wp][lane] = part;
  __syncthreads();
  if (tid < 32) {
    double v = __ldcg(a.y + (long long)I * TB + lane);
#pragma unroll
    for (int k = 0; k < BAND_THREADS / 32; ++k) v -= s.red[k][lane];
    s.d[lane] = v;
  }
  __syncthreads();
  {
    // x = U_I v: row r of U_I, columns 4q .. 4q + 3, summed over the 8
    // threads of the row
    const int r = tid / 8, q = tid % 8;
    const double* U = a.Ui + (long long)I * TB * TB + r * TB + 4 * q;
    double p = 0.0;
#pragma unroll
    for (int c = 0; c < 4; ++c) p = fma(__ldcg(U + c), s.d[4 * q + c], p);
    p += __shfl_xor_sync(0xffffffffu, p, 4);
    p += __shfl_xor_sync(0xffffffffu, p, 2);
    p += __shfl_xor_sync(0xffffffffu, p, 1);
    const long long row = (long long)I * TB + r;
    if (q == 0) {
      a.y[row] = p;
      if (row < a.n) a.sol[row] = p;
    }
  }
  w = 1;
  if (tid == 0) w = band_wait_count(a.ctr + 2, a.nb - 1 - I, &known, a.ctr + 3);
  if (!__syncthreads_and(w)) return false;
  band_publish(a.ctr + 2, a.nb - I);
  return true;
}

// The whole factorisation and both solves; launched cooperatively so that
// every block is resident.
static __global__ void __launch_bounds__(BAND_THREADS, 1) k_band_chol(BandArgs a) {
  __shared__ BandSmem s;
  for (int e = threadIdx.x; e < BAND_TRI; e += BAND_THREADS) {
    int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);  // FP32 guess, corrected below
    while ((r + 1) * (r + 2) / 2 <= e) ++r;
    while (r * (r + 1) / 2 > e) --r;
    s.tri[e] = (uint16_t)((r << 8) | (e - r * (r + 1) / 2));
  }
  const bool near = blockIdx.x < a.ncta_crit;
  const int lim = near ? a.ncrit : a.ntask;
  for (;;) {
    if (threadIdx.x == 0)
      s.task = band_load(a.ctr + 3) ? lim : (near ? 0 : a.ncrit) + atomicAdd(a.ctr + (near ? 4 : 0), 1);
    __syncthreads();
    const int q = s.task;
    __syncthreads();
    if (q >= lim) break;
    const int4 t = a.task[q];
    bool ok = true;
    switch (t.x & 7) {
      case BAND_D: ok = band_task_D(a, s, t.z); break;
      case BAND_U: ok = band_task_U(a, s, t.y, t.z, t.w, t.x >> 3); break;
      case BAND_T: ok = band_task_T(a, s, t.y, t.z); break;
      case BAND_I: ok = band_task_I(a, s, t.z); break;
      case BAND_F: ok = band_forward_task(a, s, t.z); break;
      default: ok = band_backward_task(a, s, t.z); break;
    }
    if (!ok) break;
  }
}

// Identity rows of the padding (n .. nb TB - 1) on the zeroed tiles.
static __global__ void k_band_pad(int n, int nb, int bwt, double* __restrict__ T) {
  const int R = n + blockIdx.x * blockDim.x + threadIdx.x;
  if (R >= nb * BAND_TB) return;
  const int I = R / BAND_TB;
  T[(long long)I * (bwt + 1) * (BAND_TB * BAND_TB) + (R % BAND_TB) * (BAND_TB + 1)] = 1.0;
}

// After k_band_chol: a failed factorisation (a pivot not positive or not
// finite) or a wait that ran out gives x = 0, counted; the solve's statistics.
static __global__ void k_band_finish(int n, const int* __restrict__ fail, const int* __restrict__ ctr,
                                     double* __restrict__ sol, DevState* st) {
  const bool bad = *fail != 0 || ctr[3] != 0;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (bad && i < n) sol[i] = 0.0;
  if (i == 0) {
    st->pcg_done = 1;
    st->pcg_iters = 0;
    st->pcg_rel = bad ? 1.0 : 0.0;
    if (bad) st->fallbacks += 1;
  }
}

}  // namespace ba
