// Device kernels of the LM bundle-adjustment hot path (sm_103a).
//
// Layout in HBM (T = float or double, the problem's storage precision):
//   observations are kept twice, in camera-major order (slot s, the stable
//   sort by camera) and in point-major order (slot q, the stable sort by
//   point); each order stores, per observation, the weighted Jacobian factors
//   as 18 structure-of-arrays planes of length O:
//     planes 0..5   A = sqrt(w) d pi / d X_cam          (2x3, row-major)
//     planes 6..11  B = A (-[R X]_x J_l(omega))          (2x3) = d r / d omega
//     planes 12..17 D = sqrt(w) d pi / d (f, k1, k2)     (2x3)
//   so the camera block is Jc = [B | A | D] (2x9, Sec. III-C) and the point
//   block is Jp = A R (2x3) with R from the per-camera table.  W_k = Jc^T Jp
//   is never stored: every product with it is applied in factored form.
//   Per camera: a 24-entry table (R, J_l, t, f, k1, k2), U [45] (packed upper
//   triangle of the 9x9 block), gc [9], the block-Jacobi inverse [45];
//   per point: V [6], gp [3], V*^{-1} [6], y0 = V*^{-1} gp [3].
//
// Reductions.  Every sum over observations is taken in a fixed order: a
// camera's observations are cut into pieces of at most PIECE slots, one CTA
// per piece reduces its slots (per-thread partials, warp shuffles, then the
// warps in order) and a per-camera kernel adds the pieces in order; points
// are grouped into chunks of at most CHUNK_SLOTS observations, one CTA per
// chunk computes one observation per thread into shared memory and one
// thread per point adds its observations in slot order.  No global atomics
// are used on the numeric path, so every result is bitwise reproducible.
// Per-observation arithmetic is in T; per-thread partial sums are in T; all
// cross-thread sums, dot products, costs and the gain ratio are in double.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ba.h"

namespace ba {

constexpr int PIECE = 2048;          // max camera-major slots per piece
constexpr int PIECE_THREADS = 256;
constexpr int PT_THREADS = 256;
constexpr int CAM_THREADS = 128;
constexpr int NPLANE = 18;
constexpr int CT = 24;               // camera table: R[9], Jl[9], t[3], f, k1, k2
constexpr int PART = 64;             // doubles per piece partial (54 used)
constexpr int CHUNK_SLOTS = 1024;    // max point-major slots per point chunk
constexpr int CHUNK_PTS = 1024;      // max points per point chunk
constexpr int CHUNK_THREADS = 256;

// Device-resident LM / PCG state; every field is written by exactly one
// thread of one kernel and read by later kernels.
struct DevState {
  double lam;        // damping of the next trial
  double lam_probe;  // damping for step-level calls
  double F;          // cost at the current parameters
  int cur;           // which parameter buffer holds theta
  int need_lin;      // theta changed since the last linearisation
  int pcg_done;
  int pcg_iters;
  double pcg_rel;
  int nonfinite;     // non-finite trial costs since the last stats read
  int fallbacks;     // block-Jacobi blocks replaced by diag(U*) this trial
  long long trials;
  int err;           // bit 0: index out of range, bit 1: non-finite input
  int pad;
};

__host__ __device__ constexpr int sym9(int i, int j) { return 9 * i - (i * (i - 1)) / 2 + (j - i); }
__host__ __device__ constexpr int sym3(int i, int j) { return 3 * i - (i * (i - 1)) / 2 + (j - i); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Sum NV per-thread values over the block (fixed order) and write them to out
// (NV doubles).  All threads must call it.  blockDim.x <= 256.
template <int NV>
__device__ __forceinline__ void block_sum_store(double (&v)[NV], double* __restrict__ out) {
  __shared__ double red[8][NV];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const double s = warp_sum(v[i]);
    if (lane == 0) red[warp][i] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NV; i += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w][i];
    out[i] = s;
  }
}

// Same, returning the totals to every thread instead of storing them.
template <int NV>
__device__ __forceinline__ void block_sum_all(double (&v)[NV]) {
  __shared__ double red2[8][NV];
  __shared__ double tot[NV];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const double s = warp_sum(v[i]);
    if (lane == 0) red2[warp][i] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NV; i += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red2[w][i];
    tot[i] = s;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = tot[i];
  __syncthreads();
}

// Fixed-order sum of n doubles (stride-strided) by the whole block; every
// thread gets the total.
__device__ __forceinline__ double block_sum_array(const double* __restrict__ a, int n, int stride) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += a[(long long)i * stride];
  double v[1] = {s};
  block_sum_all<1>(v);
  return v[0];
}

// ---------------------------------------------------------------------------
// SO(3) and the camera table
// ---------------------------------------------------------------------------

// R(omega) = I + a K + b K^2 and J_l(omega) = I + b K + c K^2 with K = [omega]_x,
// a = sin t / t, b = (1 - cos t)/t^2 (half-angle form 2 sin^2(t/2)/t^2),
// c = (t - sin t)/t^3; Taylor series below t = 1e-4 (a, b) and t = 0.1 (c).
__device__ inline void so3_tables(double w0, double w1, double w2, double* R, double* Jl) {
  const double t2 = w0 * w0 + w1 * w1 + w2 * w2;
  const double t = sqrt(t2);
  double a, b, c;
  if (t < 1e-4) {
    a = 1.0 - t2 / 6.0;
    b = 0.5 - t2 / 24.0;
  } else {
    const double h = sin(0.5 * t);
    a = sin(t) / t;
    b = 2.0 * h * h / t2;
  }
  if (t < 0.1) {
    c = 1.0 / 6.0 - t2 * (1.0 / 120.0 - t2 * (1.0 / 5040.0 - t2 / 362880.0));
  } else {
    c = (t - sin(t)) / (t2 * t);
  }
  // K = [[0,-w2,w1],[w2,0,-w0],[-w1,w0,0]];  K^2 = w w^T - t2 I
  const double K[9] = {0.0, -w2, w1, w2, 0.0, -w0, -w1, w0, 0.0};
  const double w[3] = {w0, w1, w2};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double K2 = w[i] * w[j] - (i == j ? t2 : 0.0);
      const double I = (i == j) ? 1.0 : 0.0;
      R[3 * i + j] = I + a * K[3 * i + j] + b * K2;
      Jl[3 * i + j] = I + b * K[3 * i + j] + c * K2;
    }
  }
}

template <typename T>
__device__ inline void camera_table(const T* __restrict__ cam, T* __restrict__ ct) {
  double R[9], Jl[9];
  so3_tables((double)cam[0], (double)cam[1], (double)cam[2], R, Jl);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    ct[i] = (T)R[i];
    ct[9 + i] = (T)Jl[i];
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) ct[18 + i] = cam[3 + i];
}

// ---------------------------------------------------------------------------
// One observation: residual, IRLS weight, weighted Jacobian factors
// ---------------------------------------------------------------------------

template <typename T>
struct Lin {
  T A[6], B[6], D[6];  // weighted factors (planes 0..17)
  T r0, r1;            // weighted residual sqrt(w) r
  T half_rho;          // 1/2 rho(|r|^2)
  T w;                 // IRLS weight rho'(|r|^2)
};

template <typename T>
__device__ __forceinline__ void project_obs(const T* __restrict__ ct, T X0, T X1, T X2,
                                            T& px, T& py, T& s) {
  const T P0 = ct[0] * X0 + ct[1] * X1 + ct[2] * X2 + ct[18];
  const T P1 = ct[3] * X0 + ct[4] * X1 + ct[5] * X2 + ct[19];
  const T P2 = ct[6] * X0 + ct[7] * X1 + ct[8] * X2 + ct[20];
  const T iz = T(1) / P2;
  px = -P0 * iz;
  py = -P1 * iz;
  const T r2 = px * px + py * py;
  s = ct[21] * (T(1) + r2 * (ct[22] + ct[23] * r2));
}

// Huber: half_rho = 1/2 rho(s), returns sqrt(w)
template <typename T>
__device__ __forceinline__ T huber_weight(T sq, T delta, T& half_rho, T& w) {
  if (delta > T(0) && sq > delta * delta) {
    const T nrm = sqrt(sq);
    half_rho = delta * nrm - T(0.5) * delta * delta;
    w = delta / nrm;
    return sqrt(w);
  }
  half_rho = T(0.5) * sq;
  w = T(1);
  return T(1);
}

template <typename T>
__device__ __forceinline__ void lin_obs(const T* __restrict__ ct, T X0, T X1, T X2, T u0, T u1,
                                        T delta, Lin<T>& o) {
  const T RX0 = ct[0] * X0 + ct[1] * X1 + ct[2] * X2;
  const T RX1 = ct[3] * X0 + ct[4] * X1 + ct[5] * X2;
  const T RX2 = ct[6] * X0 + ct[7] * X1 + ct[8] * X2;
  const T P0 = RX0 + ct[18], P1 = RX1 + ct[19], P2 = RX2 + ct[20];
  const T f = ct[21], k1 = ct[22], k2 = ct[23];
  const T iz = T(1) / P2;
  const T px = -P0 * iz, py = -P1 * iz;
  const T r2 = px * px + py * py;
  const T d = T(1) + r2 * (k1 + k2 * r2);
  const T s = f * d;
  const T r0 = s * px - u0, r1 = s * py - u1;
  T half_rho, w;
  const T sw = huber_weight(r0 * r0 + r1 * r1, delta, half_rho, w);
  o.half_rho = half_rho;
  o.w = w;
  o.r0 = sw * r0;
  o.r1 = sw * r1;
  // d pi / d p = s I + m p p^T,  m = f (2 k1 + 4 k2 |p|^2)
  const T m = f * (T(2) * k1 + T(4) * k2 * r2);
  const T a00 = s + m * px * px, a01 = m * px * py, a11 = s + m * py * py;
  // d p / d X_cam = n [[1,0,px],[0,1,py]], n = -1/P2
  const T n = -iz * sw;
  const T A0 = n * a00, A1 = n * a01, A2 = n * (a00 * px + a01 * py);
  const T A3 = n * a01, A4 = n * a11, A5 = n * (a01 * px + a11 * py);
  o.A[0] = A0; o.A[1] = A1; o.A[2] = A2; o.A[3] = A3; o.A[4] = A4; o.A[5] = A5;
  // row a of A (-[RX]_x) = RX x a ; then times J_l
  const T c0 = RX1 * A2 - RX2 * A1, c1 = RX2 * A0 - RX0 * A2, c2 = RX0 * A1 - RX1 * A0;
  const T e0 = RX1 * A5 - RX2 * A4, e1 = RX2 * A3 - RX0 * A5, e2 = RX0 * A4 - RX1 * A3;
  const T* Jl = ct + 9;
  o.B[0] = c0 * Jl[0] + c1 * Jl[3] + c2 * Jl[6];
  o.B[1] = c0 * Jl[1] + c1 * Jl[4] + c2 * Jl[7];
  o.B[2] = c0 * Jl[2] + c1 * Jl[5] + c2 * Jl[8];
  o.B[3] = e0 * Jl[0] + e1 * Jl[3] + e2 * Jl[6];
  o.B[4] = e0 * Jl[1] + e1 * Jl[4] + e2 * Jl[7];
  o.B[5] = e0 * Jl[2] + e1 * Jl[5] + e2 * Jl[8];
  // d pi / d (f, k1, k2) = (d p, f |p|^2 p, f |p|^4 p)
  const T q0 = sw * d, q1 = sw * f * r2, q2 = sw * f * r2 * r2;
  o.D[0] = q0 * px; o.D[1] = q1 * px; o.D[2] = q2 * px;
  o.D[3] = q0 * py; o.D[4] = q1 * py; o.D[5] = q2 * py;
}

// Camera row a of Jc = [B | A | D] as 9 values.
template <typename T>
__device__ __forceinline__ void jc_rows(const T* __restrict__ pl, T (&j0)[9], T (&j1)[9]) {
  j0[0] = pl[6]; j0[1] = pl[7]; j0[2] = pl[8];
  j0[3] = pl[0]; j0[4] = pl[1]; j0[5] = pl[2];
  j0[6] = pl[12]; j0[7] = pl[13]; j0[8] = pl[14];
  j1[0] = pl[9]; j1[1] = pl[10]; j1[2] = pl[11];
  j1[3] = pl[3]; j1[4] = pl[4]; j1[5] = pl[5];
  j1[6] = pl[15]; j1[7] = pl[16]; j1[8] = pl[17];
}

// Jp = A R (2x3).
template <typename T>
__device__ __forceinline__ void jp_from(const T* __restrict__ A, const T* __restrict__ R, T (&Jp)[6]) {
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Jp[3 * a + j] = A[3 * a] * R[j] + A[3 * a + 1] * R[3 + j] + A[3 * a + 2] * R[6 + j];
}

template <typename T>
__device__ __forceinline__ void load_planes(const T* __restrict__ J, long long O, long long s, T (&pl)[NPLANE]) {
#pragma unroll
  for (int p = 0; p < NPLANE; ++p) pl[p] = J[p * O + s];
}

template <typename T>
__device__ __forceinline__ void lin_to_planes(const Lin<T>& o, T (&pl)[NPLANE]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    pl[i] = o.A[i];
    pl[6 + i] = o.B[i];
    pl[12 + i] = o.D[i];
  }
}

// ---------------------------------------------------------------------------
// Set-up kernels
// ---------------------------------------------------------------------------

template <typename T>
__global__ void k_validate(int C, int P, int O, const T* __restrict__ cams, const T* __restrict__ pts,
                           const int32_t* __restrict__ ci, const int32_t* __restrict__ pi,
                           const T* __restrict__ px, DevState* st) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int bad = 0;
  if (i < O) {
    const int c = ci[i], p = pi[i];
    if (c < 0 || c >= C || p < 0 || p >= P) bad |= 1;
    if (!isfinite((double)px[2 * i]) || !isfinite((double)px[2 * i + 1])) bad |= 2;
  }
  if (i < 9LL * C && !isfinite((double)cams[i])) bad |= 2;
  if (i < 3LL * P && !isfinite((double)pts[i])) bad |= 2;
  if (bad) atomicOr(&st->err, bad);
}

// Gather the observation arrays into camera-major and point-major order.
template <typename T>
__global__ void k_gather_obs(int O, const int32_t* __restrict__ perm_cam, const int32_t* __restrict__ perm_pt,
                             const int32_t* __restrict__ ci, const int32_t* __restrict__ pi,
                             const T* __restrict__ px, int32_t* __restrict__ cm_pt, T* __restrict__ cm_px,
                             int32_t* __restrict__ pm_cam, int32_t* __restrict__ pm_pt, T* __restrict__ pm_px) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= O) return;
  const int k = perm_cam[s];
  cm_pt[s] = pi[k];
  cm_px[s] = px[2LL * k];
  cm_px[O + s] = px[2LL * k + 1];
  const int k2 = perm_pt[s];
  pm_cam[s] = ci[k2];
  pm_pt[s] = pi[k2];
  pm_px[s] = px[2LL * k2];
  pm_px[O + s] = px[2LL * k2 + 1];
}

template <typename T>
__global__ void k_project(int O, const T* __restrict__ cams, const T* __restrict__ pts,
                          const int32_t* __restrict__ ci, const int32_t* __restrict__ pi, T* __restrict__ out) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= O) return;
  T ct[CT];
  camera_table(cams + 9LL * ci[k], ct);
  const T* X = pts + 3LL * pi[k];
  T px, py, s;
  project_obs(ct, X[0], X[1], X[2], px, py, s);
  out[2 * k] = s * px;
  out[2 * k + 1] = s * py;
}

// ---------------------------------------------------------------------------
// a1 + a2: linearisation and block assembly
// ---------------------------------------------------------------------------

template <typename T>
__global__ void k_cam_prep(int C, const T* __restrict__ cams_buf, const DevState* __restrict__ st,
                           int gate, T* __restrict__ camtab) {
  if (gate && !st->need_lin) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  camera_table(cams_buf + (long long)st->cur * 9 * C + 9LL * c, camtab + (long long)CT * c);
}

// Camera-major pass: write the planes, reduce U (45), gc (9) per piece.
template <typename T>
__global__ void __launch_bounds__(PIECE_THREADS)
k_lin_cam(const int32_t* __restrict__ piece_cam, const int32_t* __restrict__ piece_beg,
          const int32_t* __restrict__ piece_end, const int32_t* __restrict__ cm_pt,
          const T* __restrict__ cm_px, const T* __restrict__ pts_buf, const T* __restrict__ camtab,
          const DevState* __restrict__ st, int gate, T delta, int O, int P, T* __restrict__ Jcm,
          double* __restrict__ part) {
  if (gate && !st->need_lin) return;
  __shared__ T sct[CT];
  const int b = blockIdx.x;
  const int c = piece_cam[b];
  if (threadIdx.x < CT) sct[threadIdx.x] = camtab[(long long)CT * c + threadIdx.x];
  __syncthreads();
  const T* pts = pts_buf + (long long)st->cur * 3 * P;
  T acc[54];
#pragma unroll
  for (int i = 0; i < 54; ++i) acc[i] = T(0);
  const int end = piece_end[b];
  for (int s = piece_beg[b] + threadIdx.x; s < end; s += PIECE_THREADS) {
    const int j = cm_pt[s];
    Lin<T> o;
    lin_obs(sct, pts[3LL * j], pts[3LL * j + 1], pts[3LL * j + 2], cm_px[s], cm_px[(long long)O + s], delta, o);
    T pl[NPLANE];
    lin_to_planes(o, pl);
#pragma unroll
    for (int p = 0; p < NPLANE; ++p) Jcm[(long long)p * O + s] = pl[p];
    T j0[9], j1[9];
    jc_rows(pl, j0, j1);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
#pragma unroll
      for (int k = i; k < 9; ++k) acc[sym9(i, k)] += j0[i] * j0[k] + j1[i] * j1[k];
      acc[45 + i] += j0[i] * o.r0 + j1[i] * o.r1;
    }
  }
  double v[54];
#pragma unroll
  for (int i = 0; i < 54; ++i) v[i] = (double)acc[i];
  block_sum_store<54>(v, part + (long long)PART * b);
}

// Add the pieces of each camera in order: U [C][45], gc [C][9].
__global__ void k_cam_combine_lin(int C, const int32_t* __restrict__ cam_piece_ptr,
                                  const double* __restrict__ part, const DevState* __restrict__ st,
                                  int gate, double* __restrict__ U, double* __restrict__ gc) {
  if (gate && !st->need_lin) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const int p0 = cam_piece_ptr[c], p1 = cam_piece_ptr[c + 1];
  for (int i = 0; i < 54; ++i) {
    double s = 0.0;
    for (int p = p0; p < p1; ++p) s += part[(long long)PART * p + i];
    if (i < 45) U[45LL * c + i] = s;
    else gc[9LL * c + i - 45] = s;
  }
}

// Point-major pass over one chunk of points: write the planes, V (6) and
// gp (3) per point.  One thread per observation (coalesced plane stores);
// each observation's 9 contributions go to shared memory and one thread per
// point adds its observations in slot order.  A point with more than
// CHUNK_SLOTS observations is a chunk of its own and is reduced by the block.
template <typename T>
__device__ __forceinline__ void lin_pt_obs(int q, int O, const int32_t* __restrict__ pm_cam,
                                           const int32_t* __restrict__ pm_pt, const T* __restrict__ pm_px,
                                           const T* __restrict__ pts, const T* __restrict__ camtab, T delta,
                                           T* __restrict__ Jpm, T (&v)[9]) {
  const int j = pm_pt[q];
  const T* ct = camtab + (long long)CT * pm_cam[q];
  T ctl[CT];
#pragma unroll
  for (int i = 0; i < CT; ++i) ctl[i] = ct[i];
  Lin<T> o;
  lin_obs(ctl, pts[3LL * j], pts[3LL * j + 1], pts[3LL * j + 2], pm_px[q], pm_px[(long long)O + q], delta, o);
  T pl[NPLANE];
  lin_to_planes(o, pl);
#pragma unroll
  for (int p = 0; p < NPLANE; ++p) Jpm[(long long)p * O + q] = pl[p];
  T Jp[6];
  jp_from(o.A, ctl, Jp);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = a; b < 3; ++b) v[sym3(a, b)] = Jp[a] * Jp[b] + Jp[3 + a] * Jp[3 + b];
    v[6 + a] = Jp[a] * o.r0 + Jp[3 + a] * o.r1;
  }
}

template <typename T>
__global__ void __launch_bounds__(CHUNK_THREADS)
k_lin_pt(const int32_t* __restrict__ pchunk, int O, const int32_t* __restrict__ rowptr_pt,
         const int32_t* __restrict__ pm_cam, const int32_t* __restrict__ pm_pt, const T* __restrict__ pm_px,
         const T* __restrict__ pts_buf, const T* __restrict__ camtab, const DevState* __restrict__ st, int P,
         int gate, T delta, T* __restrict__ Jpm, double* __restrict__ V, double* __restrict__ gp) {
  if (gate && !st->need_lin) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sv = reinterpret_cast<T*>(smem_raw);  // [CHUNK_SLOTS][9]
  const T* pts = pts_buf + (long long)st->cur * 3 * P;
  const int j0 = pchunk[blockIdx.x], j1 = pchunk[blockIdx.x + 1];
  const int s0 = rowptr_pt[j0], s1 = rowptr_pt[j1];
  if (s1 - s0 <= CHUNK_SLOTS) {
    for (int q = s0 + threadIdx.x; q < s1; q += CHUNK_THREADS) {
      T v[9];
      lin_pt_obs(q, O, pm_cam, pm_pt, pm_px, pts, camtab, delta, Jpm, v);
#pragma unroll
      for (int i = 0; i < 9; ++i) sv[(q - s0) * 9 + i] = v[i];
    }
    __syncthreads();
    for (int j = j0 + threadIdx.x; j < j1; j += CHUNK_THREADS) {
      T acc[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) acc[i] = T(0);
      const int q1 = rowptr_pt[j + 1];
      for (int q = rowptr_pt[j]; q < q1; ++q)
#pragma unroll
        for (int i = 0; i < 9; ++i) acc[i] += sv[(q - s0) * 9 + i];
#pragma unroll
      for (int i = 0; i < 6; ++i) V[6LL * j + i] = (double)acc[i];
#pragma unroll
      for (int i = 0; i < 3; ++i) gp[3LL * j + i] = (double)acc[6 + i];
    }
  } else {
    T acc[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) acc[i] = T(0);
    for (int q = s0 + threadIdx.x; q < s1; q += CHUNK_THREADS) {
      T v[9];
      lin_pt_obs(q, O, pm_cam, pm_pt, pm_px, pts, camtab, delta, Jpm, v);
#pragma unroll
      for (int i = 0; i < 9; ++i) acc[i] += v[i];
    }
    double d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = (double)acc[i];
    block_sum_all<9>(d);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int i = 0; i < 6; ++i) V[6LL * j0 + i] = d[i];
#pragma unroll
      for (int i = 0; i < 3; ++i) gp[3LL * j0 + i] = d[6 + i];
    }
  }
}

// ---------------------------------------------------------------------------
// a3: damping, V*^{-1}, Schur right-hand side and block-Jacobi blocks
// ---------------------------------------------------------------------------

__device__ __forceinline__ double damp(double d, double lam, double dmin, double dmax) {
  return lam * fmin(fmax(d, dmin), dmax);
}

// V*_j = V_j + lam clamp(diag V_j);  Vinv = V*^{-1};  y0 = Vinv gp.
template <typename T>
__global__ void k_pt_damp(int P, const double* __restrict__ V, const double* __restrict__ gp,
                          const double* __restrict__ lam_ptr, double dmin, double dmax,
                          T* __restrict__ Vinv, T* __restrict__ y0) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P) return;
  const double lam = *lam_ptr;
  const double* v = V + 6LL * j;
  const double a = v[0] + damp(v[0], lam, dmin, dmax), b = v[1], c = v[2];
  const double d = v[3] + damp(v[3], lam, dmin, dmax), e = v[4];
  const double f = v[5] + damp(v[5], lam, dmin, dmax);
  const double A00 = d * f - e * e, A01 = c * e - b * f, A02 = b * e - c * d;
  const double A11 = a * f - c * c, A12 = b * c - a * e, A22 = a * d - b * b;
  const double det = a * A00 + b * A01 + c * A02;
  const double id = 1.0 / det;
  const double inv[6] = {A00 * id, A01 * id, A02 * id, A11 * id, A12 * id, A22 * id};
#pragma unroll
  for (int i = 0; i < 6; ++i) Vinv[6LL * j + i] = (T)inv[i];
  const double g0 = gp[3LL * j], g1 = gp[3LL * j + 1], g2 = gp[3LL * j + 2];
  y0[3LL * j] = (T)(inv[0] * g0 + inv[1] * g1 + inv[2] * g2);
  y0[3LL * j + 1] = (T)(inv[1] * g0 + inv[3] * g1 + inv[4] * g2);
  y0[3LL * j + 2] = (T)(inv[2] * g0 + inv[4] * g1 + inv[5] * g2);
}

// Camera-major pass: per piece, sum_k Jc^T (Jp V*^{-1} Jp^T) Jc (45) and
// sum_k Jc^T Jp y0 (9).
template <typename T>
__global__ void __launch_bounds__(PIECE_THREADS)
k_schur_cam(const int32_t* __restrict__ piece_cam, const int32_t* __restrict__ piece_beg,
            const int32_t* __restrict__ piece_end, const int32_t* __restrict__ cm_pt,
            const T* __restrict__ Jcm, const T* __restrict__ camtab, const T* __restrict__ Vinv,
            const T* __restrict__ y0, int O, double* __restrict__ part) {
  __shared__ T sR[9];
  const int b = blockIdx.x;
  const int c = piece_cam[b];
  if (threadIdx.x < 9) sR[threadIdx.x] = camtab[(long long)CT * c + threadIdx.x];
  __syncthreads();
  T acc[54];
#pragma unroll
  for (int i = 0; i < 54; ++i) acc[i] = T(0);
  const int end = piece_end[b];
  for (int s = piece_beg[b] + threadIdx.x; s < end; s += PIECE_THREADS) {
    const int j = cm_pt[s];
    T pl[NPLANE];
    load_planes(Jcm, O, s, pl);
    T Jp[6];
    jp_from(pl, sR, Jp);
    const T* vi = Vinv + 6LL * j;
    const T v00 = vi[0], v01 = vi[1], v02 = vi[2], v11 = vi[3], v12 = vi[4], v22 = vi[5];
    // T2 = Jp Vinv (2x3)
    T t[6];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      t[3 * a] = Jp[3 * a] * v00 + Jp[3 * a + 1] * v01 + Jp[3 * a + 2] * v02;
      t[3 * a + 1] = Jp[3 * a] * v01 + Jp[3 * a + 1] * v11 + Jp[3 * a + 2] * v12;
      t[3 * a + 2] = Jp[3 * a] * v02 + Jp[3 * a + 1] * v12 + Jp[3 * a + 2] * v22;
    }
    const T m00 = t[0] * Jp[0] + t[1] * Jp[1] + t[2] * Jp[2];
    const T m01 = t[0] * Jp[3] + t[1] * Jp[4] + t[2] * Jp[5];
    const T m11 = t[3] * Jp[3] + t[4] * Jp[4] + t[5] * Jp[5];
    const T* yy = y0 + 3LL * j;
    const T y00 = yy[0], y01 = yy[1], y02 = yy[2];
    const T e0 = Jp[0] * y00 + Jp[1] * y01 + Jp[2] * y02;
    const T e1 = Jp[3] * y00 + Jp[4] * y01 + Jp[5] * y02;
    T j0[9], j1[9];
    jc_rows(pl, j0, j1);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const T n0 = m00 * j0[i] + m01 * j1[i];
      const T n1 = m01 * j0[i] + m11 * j1[i];
#pragma unroll
      for (int k = i; k < 9; ++k) acc[sym9(i, k)] += n0 * j0[k] + n1 * j1[k];
      acc[45 + i] += j0[i] * e0 + j1[i] * e1;
    }
  }
  double v[54];
#pragma unroll
  for (int i = 0; i < 54; ++i) v[i] = (double)acc[i];
  block_sum_store<54>(v, part + (long long)PART * b);
}

// In-place Cholesky of a packed symmetric 9x9 (upper triangle, sym9) and its
// inverse, in double.  Returns false if a pivot is not positive/finite.
__device__ inline bool spd_inverse9(const double* __restrict__ S, double* __restrict__ Minv) {
  double L[9][9];
#pragma unroll
  for (int i = 0; i < 9; ++i)
#pragma unroll
    for (int j = 0; j < 9; ++j) L[i][j] = 0.0;
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    double d = S[sym9(j, j)];
#pragma unroll
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    if (!(d > 0.0) || !isfinite(d)) return false;
    const double ljj = sqrt(d);
    L[j][j] = ljj;
    const double il = 1.0 / ljj;
#pragma unroll
    for (int i = j + 1; i < 9; ++i) {
      double s = S[sym9(j, i)];
#pragma unroll
      for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
      L[i][j] = s * il;
    }
  }
  // Linv lower triangular: Linv = L^{-1}
  double Li[9][9];
#pragma unroll
  for (int i = 0; i < 9; ++i)
#pragma unroll
    for (int j = 0; j < 9; ++j) Li[i][j] = 0.0;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    Li[i][i] = 1.0 / L[i][i];
#pragma unroll
    for (int j = 0; j < i; ++j) {
      double s = 0.0;
#pragma unroll
      for (int k = j; k < i; ++k) s += L[i][k] * Li[k][j];
      Li[i][j] = -s * Li[i][i];
    }
  }
  // M = Linv^T Linv
#pragma unroll
  for (int i = 0; i < 9; ++i)
#pragma unroll
    for (int j = i; j < 9; ++j) {
      double s = 0.0;
#pragma unroll
      for (int k = j; k < 9; ++k) s += Li[k][i] * Li[k][j];
      Minv[sym9(i, j)] = s;
    }
  return true;
}

__device__ __forceinline__ void sym9_matvec(const double* __restrict__ M, const double* __restrict__ x,
                                            double* __restrict__ y) {
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 9; ++j) s += M[i <= j ? sym9(i, j) : sym9(j, i)] * x[j];
    y[i] = s;
  }
}

// U*_i x_i with U* = U + lam clamp(diag U).
__device__ __forceinline__ void ustar_matvec(const double* __restrict__ U, double lam, double dmin, double dmax,
                                             const double* __restrict__ x, double* __restrict__ y) {
  sym9_matvec(U, x, y);
#pragma unroll
  for (int i = 0; i < 9; ++i) y[i] += damp(U[sym9(i, i)], lam, dmin, dmax) * x[i];
}

// Per camera: S_ii, b_i, M_i = S_ii^{-1}; PCG start x = 0, r = b, z = M r,
// p = z; per-block partial sums of r.z and b.b.
template <typename T>
__global__ void __launch_bounds__(CAM_THREADS)
k_cam_combine_schur(int C, const int32_t* __restrict__ cam_piece_ptr, const double* __restrict__ part,
                    const double* __restrict__ U, const double* __restrict__ gc,
                    const double* __restrict__ lam_ptr, double dmin, double dmax, double* __restrict__ Minv,
                    double* __restrict__ x, double* __restrict__ r, double* __restrict__ z,
                    double* __restrict__ p, T* __restrict__ pT, double* __restrict__ dot_rz1,
                    double* __restrict__ dot_bb, DevState* st) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double rz = 0.0, bb = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->pcg_done = 0;
    st->pcg_iters = 0;
    st->pcg_rel = 1.0;
    st->fallbacks = 0;
  }
  if (c < C) {
    const double lam = *lam_ptr;
    const int p0 = cam_piece_ptr[c], p1 = cam_piece_ptr[c + 1];
    double S[45], bv[9];
    const double* Uc = U + 45LL * c;
#pragma unroll
    for (int i = 0; i < 45; ++i) S[i] = Uc[i];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      S[sym9(i, i)] += damp(Uc[sym9(i, i)], lam, dmin, dmax);
      bv[i] = -gc[9LL * c + i];
    }
    for (int q = p0; q < p1; ++q) {
      const double* pp = part + (long long)PART * q;
#pragma unroll
      for (int i = 0; i < 45; ++i) S[i] -= pp[i];
#pragma unroll
      for (int i = 0; i < 9; ++i) bv[i] += pp[45 + i];
    }
    double M[45];
    if (!spd_inverse9(S, M)) {
      // not SPD in this precision: fall back to the inverse diagonal of U*
#pragma unroll
      for (int i = 0; i < 45; ++i) M[i] = 0.0;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const double d = Uc[sym9(i, i)] + damp(Uc[sym9(i, i)], lam, dmin, dmax);
        M[sym9(i, i)] = 1.0 / d;
      }
      atomicAdd(&st->fallbacks, 1);
    }
#pragma unroll
    for (int i = 0; i < 45; ++i) Minv[45LL * c + i] = M[i];
    double zz[9];
    sym9_matvec(M, bv, zz);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      x[9LL * c + i] = 0.0;
      r[9LL * c + i] = bv[i];
      z[9LL * c + i] = zz[i];
      p[9LL * c + i] = zz[i];
      pT[9LL * c + i] = (T)zz[i];
      rz += bv[i] * zz[i];
      bb += bv[i] * bv[i];
    }
  }
  double v[2] = {rz, bb};
  block_sum_all<2>(v);
  if (threadIdx.x == 0) {
    dot_rz1[blockIdx.x] = v[0];
    dot_bb[blockIdx.x] = v[1];
  }
}

// ---------------------------------------------------------------------------
// a4: PCG iteration k (S p through two passes, then the vector updates)
// ---------------------------------------------------------------------------

// Pass A (point-major): t_j = V*_j^{-1} sum_{k in pt j} Jp_k^T (Jc_k p_c(k)),
// over one chunk of points (thread per observation, shared-memory segmented
// sum per point as in k_lin_pt).  With MODE 1 (back-substitution) it forms
// dp_j = -(y0_j + t_j), writes the trial point theta_p + dp_j and reduces
// gp_j . dp_j per chunk.
template <typename T>
__device__ __forceinline__ void pass_a_obs(int q, long long O, const int32_t* __restrict__ pm_cam,
                                           const T* __restrict__ Jpm, const T* __restrict__ camtab,
                                           const T* __restrict__ xc, T& z0, T& z1, T& z2) {
  const int c = pm_cam[q];
  T pl[NPLANE];
  load_planes(Jpm, O, q, pl);
  const T* xv = xc + 9LL * c;
  T j0[9], j1[9];
  jc_rows(pl, j0, j1);
  T e0 = 0, e1 = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const T xi = xv[i];
    e0 += j0[i] * xi;
    e1 += j1[i] * xi;
  }
  const T a0 = pl[0] * e0 + pl[3] * e1;
  const T a1 = pl[1] * e0 + pl[4] * e1;
  const T a2 = pl[2] * e0 + pl[5] * e1;
  const T* R = camtab + (long long)CT * c;
  z0 = R[0] * a0 + R[3] * a1 + R[6] * a2;
  z1 = R[1] * a0 + R[4] * a1 + R[7] * a2;
  z2 = R[2] * a0 + R[5] * a1 + R[8] * a2;
}

template <typename T, int MODE>
__device__ __forceinline__ double pass_a_point(int j, int P, T z0, T z1, T z2, const T* __restrict__ Vinv,
                                               T* __restrict__ out, const T* __restrict__ y0,
                                               const double* __restrict__ gp, T* __restrict__ pts_buf, int cur) {
  const T* vi = Vinv + 6LL * j;
  const T t0 = vi[0] * z0 + vi[1] * z1 + vi[2] * z2;
  const T t1 = vi[1] * z0 + vi[3] * z1 + vi[4] * z2;
  const T t2 = vi[2] * z0 + vi[4] * z1 + vi[5] * z2;
  if (MODE == 0) {
    out[3LL * j] = t0;
    out[3LL * j + 1] = t1;
    out[3LL * j + 2] = t2;
    return 0.0;
  }
  const T d0 = -(y0[3LL * j] + t0), d1 = -(y0[3LL * j + 1] + t1), d2 = -(y0[3LL * j + 2] + t2);
  out[3LL * j] = d0;
  out[3LL * j + 1] = d1;
  out[3LL * j + 2] = d2;
  const T* src = pts_buf + (long long)cur * 3 * P + 3LL * j;
  T* dst = pts_buf + (long long)(1 - cur) * 3 * P + 3LL * j;
  dst[0] = src[0] + d0;
  dst[1] = src[1] + d1;
  dst[2] = src[2] + d2;
  return gp[3LL * j] * (double)d0 + gp[3LL * j + 1] * (double)d1 + gp[3LL * j + 2] * (double)d2;
}

template <typename T, int MODE>
__global__ void __launch_bounds__(CHUNK_THREADS)
k_pass_a(const int32_t* __restrict__ pchunk, int P, int O, const int32_t* __restrict__ rowptr_pt,
         const int32_t* __restrict__ pm_cam, const T* __restrict__ Jpm, const T* __restrict__ camtab,
         const T* __restrict__ xc, const T* __restrict__ Vinv, const DevState* __restrict__ st, int check_done,
         T* __restrict__ out, const T* __restrict__ y0, const double* __restrict__ gp, T* __restrict__ pts_buf,
         double* __restrict__ dot_gp) {
  if (MODE == 0 && check_done && st->pcg_done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sz = reinterpret_cast<T*>(smem_raw);  // [CHUNK_SLOTS][3]
  const int cur = MODE == 1 ? st->cur : 0;
  const int j0 = pchunk[blockIdx.x], j1 = pchunk[blockIdx.x + 1];
  const int s0 = rowptr_pt[j0], s1 = rowptr_pt[j1];
  double gd = 0.0;
  if (s1 - s0 <= CHUNK_SLOTS) {
    for (int q = s0 + threadIdx.x; q < s1; q += CHUNK_THREADS) {
      T z0, z1, z2;
      pass_a_obs(q, O, pm_cam, Jpm, camtab, xc, z0, z1, z2);
      sz[(q - s0) * 3] = z0;
      sz[(q - s0) * 3 + 1] = z1;
      sz[(q - s0) * 3 + 2] = z2;
    }
    __syncthreads();
    for (int j = j0 + threadIdx.x; j < j1; j += CHUNK_THREADS) {
      T z0 = 0, z1 = 0, z2 = 0;
      const int q1 = rowptr_pt[j + 1];
      for (int q = rowptr_pt[j]; q < q1; ++q) {
        z0 += sz[(q - s0) * 3];
        z1 += sz[(q - s0) * 3 + 1];
        z2 += sz[(q - s0) * 3 + 2];
      }
      gd += pass_a_point<T, MODE>(j, P, z0, z1, z2, Vinv, out, y0, gp, pts_buf, cur);
    }
  } else {
    T z0 = 0, z1 = 0, z2 = 0;
    for (int q = s0 + threadIdx.x; q < s1; q += CHUNK_THREADS) {
      T a0, a1, a2;
      pass_a_obs(q, O, pm_cam, Jpm, camtab, xc, a0, a1, a2);
      z0 += a0;
      z1 += a1;
      z2 += a2;
    }
    double d[3] = {(double)z0, (double)z1, (double)z2};
    block_sum_all<3>(d);
    if (threadIdx.x == 0) gd = pass_a_point<T, MODE>(j0, P, (T)d[0], (T)d[1], (T)d[2], Vinv, out, y0, gp, pts_buf, cur);
  }
  if (MODE == 1) {
    double v[1] = {gd};
    block_sum_all<1>(v);
    if (threadIdx.x == 0) dot_gp[blockIdx.x] = v[0];
  }
}

// Pass B (camera-major): per piece, sum_k Jc_k^T (Jp_k t_p(k)) (9 values).
template <typename T>
__global__ void __launch_bounds__(PIECE_THREADS)
k_pass_b(const int32_t* __restrict__ piece_cam, const int32_t* __restrict__ piece_beg,
         const int32_t* __restrict__ piece_end, const int32_t* __restrict__ cm_pt,
         const T* __restrict__ Jcm, const T* __restrict__ camtab, const T* __restrict__ tpt,
         const DevState* __restrict__ st, int check_done, int O, double* __restrict__ part) {
  if (check_done && st->pcg_done) return;
  __shared__ T sR[9];
  const int b = blockIdx.x;
  const int c = piece_cam[b];
  if (threadIdx.x < 9) sR[threadIdx.x] = camtab[(long long)CT * c + threadIdx.x];
  __syncthreads();
  T acc[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) acc[i] = T(0);
  const int end = piece_end[b];
#pragma unroll 4
  for (int s = piece_beg[b] + threadIdx.x; s < end; s += PIECE_THREADS) {
    const int j = cm_pt[s];
    T pl[NPLANE];
    load_planes(Jcm, O, s, pl);
    const T t0 = tpt[3LL * j], t1 = tpt[3LL * j + 1], t2 = tpt[3LL * j + 2];
    const T g0 = sR[0] * t0 + sR[1] * t1 + sR[2] * t2;
    const T g1 = sR[3] * t0 + sR[4] * t1 + sR[5] * t2;
    const T g2 = sR[6] * t0 + sR[7] * t1 + sR[8] * t2;
    const T h0 = pl[0] * g0 + pl[1] * g1 + pl[2] * g2;
    const T h1 = pl[3] * g0 + pl[4] * g1 + pl[5] * g2;
    T j0[9], j1[9];
    jc_rows(pl, j0, j1);
#pragma unroll
    for (int i = 0; i < 9; ++i) acc[i] += j0[i] * h0 + j1[i] * h1;
  }
  double v[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) v[i] = (double)acc[i];
  block_sum_store<9>(v, part + (long long)PART * b);
}

// q = U* p - sum of pass-B pieces; per-block partial p.q.
__global__ void __launch_bounds__(CAM_THREADS)
k_pcg_q(int C, const int32_t* __restrict__ cam_piece_ptr, const double* __restrict__ part,
        const double* __restrict__ U, const double* __restrict__ lam_ptr, double dmin, double dmax,
        const double* __restrict__ p, double* __restrict__ q, double* __restrict__ dot_pq,
        const DevState* __restrict__ st, int check_done) {
  if (check_done && st->pcg_done) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double pq = 0.0;
  if (c < C) {
    const double lam = *lam_ptr;
    double pv[9], y[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) pv[i] = p[9LL * c + i];
    ustar_matvec(U + 45LL * c, lam, dmin, dmax, pv, y);
    const int p0 = cam_piece_ptr[c], p1 = cam_piece_ptr[c + 1];
    for (int k = p0; k < p1; ++k) {
#pragma unroll
      for (int i = 0; i < 9; ++i) y[i] -= part[(long long)PART * k + i];
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      q[9LL * c + i] = y[i];
      pq += pv[i] * y[i];
    }
  }
  double v[1] = {pq};
  block_sum_all<1>(v);
  if (threadIdx.x == 0 && dot_pq) dot_pq[blockIdx.x] = v[0];
}

// alpha = (r.z)_old / p.q; x += alpha p; r -= alpha q; z = M r;
// partial r.z into dot_rz[k & 1], partial r.r.
__global__ void __launch_bounds__(CAM_THREADS)
k_pcg_update(int C, int nb, int k, const double* __restrict__ dot_pq, double* __restrict__ dot_rz,
             double* __restrict__ dot_rr, const double* __restrict__ p, const double* __restrict__ q,
             double* __restrict__ x, double* __restrict__ r, double* __restrict__ z,
             const double* __restrict__ Minv, DevState* st) {
  if (st->pcg_done) return;
  const double pq = block_sum_array(dot_pq, nb, 1);
  const double rz_old = block_sum_array(dot_rz + ((k + 1) & 1) * nb, nb, 1);
  if (!(pq > 0.0) || !isfinite(pq)) {
    // no positive curvature (b = 0 or breakdown): keep x, stop
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st->pcg_done = 1;
      st->pcg_iters = k;
      if (k == 0) st->pcg_rel = 0.0;
    }
    return;
  }
  const double alpha = rz_old / pq;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double rz = 0.0, rr = 0.0;
  if (c < C) {
    double rv[9], zz[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      x[9LL * c + i] += alpha * p[9LL * c + i];
      rv[i] = r[9LL * c + i] - alpha * q[9LL * c + i];
      r[9LL * c + i] = rv[i];
    }
    sym9_matvec(Minv + 45LL * c, rv, zz);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      z[9LL * c + i] = zz[i];
      rz += rv[i] * zz[i];
      rr += rv[i] * rv[i];
    }
  }
  double v[2] = {rz, rr};
  block_sum_all<2>(v);
  if (threadIdx.x == 0) {
    dot_rz[(k & 1) * nb + blockIdx.x] = v[0];
    dot_rr[blockIdx.x] = v[1];
  }
}

// Convergence test |r| <= tol |b|; beta = (r.z)_new / (r.z)_old; p = z + beta p.
template <typename T>
__global__ void __launch_bounds__(CAM_THREADS)
k_pcg_direction(int C, int nb, int k, double tol, const double* __restrict__ dot_rz,
                const double* __restrict__ dot_rr, const double* __restrict__ dot_bb,
                const double* __restrict__ z, double* __restrict__ p, T* __restrict__ pT, DevState* st) {
  if (st->pcg_done) return;
  const double rz_new = block_sum_array(dot_rz + (k & 1) * nb, nb, 1);
  const double rz_old = block_sum_array(dot_rz + ((k + 1) & 1) * nb, nb, 1);
  const double rr = block_sum_array(dot_rr, nb, 1);
  const double bb = block_sum_array(dot_bb, nb, 1);
  const bool conv = sqrt(rr) <= tol * sqrt(bb);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->pcg_iters = k + 1;
    st->pcg_rel = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    if (conv) st->pcg_done = 1;
  }
  if (conv) return;
  const double beta = rz_new / rz_old;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < C) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const double pv = z[9LL * c + i] + beta * p[9LL * c + i];
      p[9LL * c + i] = pv;
      pT[9LL * c + i] = (T)pv;
    }
  }
}

// ---------------------------------------------------------------------------
// a5 / a6: trial parameters, trial cost, model reduction, LM control
// ---------------------------------------------------------------------------

// Trial cameras theta_c + dc, dc in T, partial gc . dc.
template <typename T>
__global__ void __launch_bounds__(CAM_THREADS)
k_cam_trial(int C, const double* __restrict__ x, const double* __restrict__ gc, T* __restrict__ cams_buf,
            const DevState* __restrict__ st, T* __restrict__ xT, double* __restrict__ dot_gc) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double gd = 0.0;
  if (c < C) {
    const int cur = st->cur;
    const T* src = cams_buf + (long long)cur * 9 * C + 9LL * c;
    T* dst = cams_buf + (long long)(1 - cur) * 9 * C + 9LL * c;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const T d = (T)x[9LL * c + i];
      xT[9LL * c + i] = d;
      dst[i] = src[i] + d;
      gd += gc[9LL * c + i] * (double)d;
    }
  }
  double v[1] = {gd};
  block_sum_all<1>(v);
  if (threadIdx.x == 0) dot_gc[blockIdx.x] = v[0];
}

// Camera-major pass over the pieces: cost 1/2 sum rho at the parameters in
// buffer (which == 0: current, 1: trial), and with MODEL the quadratic term
// sum_k |Jc_k dc + Jp_k dp|^2 of the model reduction (weights folded in).
template <typename T, bool MODEL>
__global__ void __launch_bounds__(PIECE_THREADS)
k_cost_cam(const int32_t* __restrict__ piece_cam, const int32_t* __restrict__ piece_beg,
           const int32_t* __restrict__ piece_end, const int32_t* __restrict__ cm_pt,
           const T* __restrict__ cm_px, const T* __restrict__ cams_buf, const T* __restrict__ pts_buf,
           const DevState* __restrict__ st, int which, T delta, int C, int P, int O,
           const T* __restrict__ Jcm, const T* __restrict__ camtab, const T* __restrict__ xT,
           const T* __restrict__ dp, double* __restrict__ part) {
  __shared__ T sct[CT];
  __shared__ T sR[9];
  __shared__ T sdc[9];
  const int b = blockIdx.x;
  const int c = piece_cam[b];
  const int buf = which ? 1 - st->cur : st->cur;
  if (threadIdx.x == 0) camera_table(cams_buf + (long long)buf * 9 * C + 9LL * c, sct);
  if (MODEL && threadIdx.x >= 32 && threadIdx.x < 41) sR[threadIdx.x - 32] = camtab[(long long)CT * c + threadIdx.x - 32];
  if (MODEL && threadIdx.x >= 64 && threadIdx.x < 73) sdc[threadIdx.x - 64] = xT[9LL * c + threadIdx.x - 64];
  __syncthreads();
  const T* pts = pts_buf + (long long)buf * 3 * P;
  double cost = 0.0, quad = 0.0;
  const int end = piece_end[b];
  for (int s = piece_beg[b] + threadIdx.x; s < end; s += PIECE_THREADS) {
    const int j = cm_pt[s];
    T px, py, sc;
    project_obs(sct, pts[3LL * j], pts[3LL * j + 1], pts[3LL * j + 2], px, py, sc);
    const T r0 = sc * px - cm_px[s], r1 = sc * py - cm_px[(long long)O + s];
    T hr, w;
    huber_weight(r0 * r0 + r1 * r1, delta, hr, w);
    cost += (double)hr;
    if (MODEL) {
      T pl[NPLANE];
      load_planes(Jcm, O, s, pl);
      T j0[9], j1[9];
      jc_rows(pl, j0, j1);
      T Jp[6];
      jp_from(pl, sR, Jp);
      const T d0 = dp[3LL * j], d1 = dp[3LL * j + 1], d2 = dp[3LL * j + 2];
      T e0 = Jp[0] * d0 + Jp[1] * d1 + Jp[2] * d2;
      T e1 = Jp[3] * d0 + Jp[4] * d1 + Jp[5] * d2;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        e0 += j0[i] * sdc[i];
        e1 += j1[i] * sdc[i];
      }
      quad += (double)e0 * (double)e0 + (double)e1 * (double)e1;
    }
  }
  double v[2] = {cost, quad};
  block_sum_store<2>(v, part + (long long)PART * b);
}

// Sum the cost pieces into st->F (initial cost / after set_params).
__global__ void k_cost_finalize(int npieces, const double* __restrict__ part, DevState* st) {
  const double F = block_sum_array(part, npieces, PART);
  if (threadIdx.x == 0) {
    st->F = F;
    if (!isfinite(F)) st->err |= 2;
  }
}

// Gain ratio, accept / reject and the damping update (one block).
__global__ void k_lm_control(int npieces, const double* __restrict__ part, int ncb,
                             const double* __restrict__ dot_gc, int npb, const double* __restrict__ dot_gp,
                             double up, double down, double rho_good, double rho_bad, double lam_min,
                             double lam_max, DevState* st, ba_iter_stats* __restrict__ stats, int cap) {
  const double Ft = block_sum_array(part, npieces, PART);
  const double quad = block_sum_array(part + 1, npieces, PART);
  const double lin = block_sum_array(dot_gc, ncb, 1) + block_sum_array(dot_gp, npb, 1);
  if (threadIdx.x != 0) return;
  const double F = st->F;
  const double lam = st->lam;
  const double model = -lin - 0.5 * quad;
  const double rho = model != 0.0 ? (F - Ft) / model : nan("");
  const bool finite = isfinite(Ft);
  const bool accept = finite && model > 0.0 && Ft < F;
  const long long t = st->trials;
  ba_iter_stats& sr = stats[t % cap];
  sr.cost = F;
  sr.cost_trial = Ft;
  sr.model = model;
  sr.rho = rho;
  sr.lambda = lam;
  sr.pcg_rel_res = st->pcg_rel;
  sr.accepted = accept ? 1 : 0;
  sr.pcg_iters = st->pcg_iters;
  sr.precond_fallbacks = st->fallbacks;
  sr.reserved = 0;
  if (!finite) st->nonfinite += 1;
  double nl = lam;
  if (accept) {
    st->cur = 1 - st->cur;
    st->F = Ft;
    st->need_lin = 1;
    if (rho > rho_good) nl = fmax(lam / up, lam_min);
    else if (rho < rho_bad) nl = fmin(lam / down, lam_max);
  } else {
    st->need_lin = 0;
    nl = fmin(lam / down, lam_max);
  }
  st->lam = nl;
  st->trials = t + 1;
}

// ---------------------------------------------------------------------------
// Step-level helpers
// ---------------------------------------------------------------------------

template <typename T>
__global__ void k_cast_vec(long long n, const double* __restrict__ a, T* __restrict__ b) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (T)a[i];
}

// Unpack U [C][45] to [C][9][9] (or V [P][6] to [P][3][3]).
__global__ void k_unpack_sym(long long n, int dim, const double* __restrict__ packed, double* __restrict__ full) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * dim * dim) return;
  const long long blk = i / (dim * dim);
  const int rc = (int)(i % (dim * dim));
  int a = rc / dim, b = rc % dim;
  if (a > b) {
    const int t = a;
    a = b;
    b = t;
  }
  const int np = dim * (dim + 1) / 2;
  const int idx = dim * a - (a * (a - 1)) / 2 + (b - a);
  full[i] = packed[blk * np + idx];
}

// Export sqrt(w) Jc [O][2][9], sqrt(w) Jp [O][2][3] (from the camera-major
// planes) and w [O] in input order.
template <typename T>
__global__ void k_export_lin(int O, int P, const int32_t* __restrict__ perm_cam, const int32_t* __restrict__ ci,
                             const int32_t* __restrict__ cm_pt, const T* __restrict__ cm_px,
                             const T* __restrict__ Jcm, const T* __restrict__ camtab,
                             const T* __restrict__ pts_buf, const DevState* __restrict__ st, T delta,
                             T* __restrict__ Jc, T* __restrict__ Jp, T* __restrict__ w) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= O) return;
  const long long k = perm_cam[s];
  const int c = ci[k];
  const T* ct = camtab + (long long)CT * c;
  T pl[NPLANE];
  load_planes(Jcm, O, s, pl);
  if (Jc) {
    T j0[9], j1[9];
    jc_rows(pl, j0, j1);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      Jc[18 * k + i] = j0[i];
      Jc[18 * k + 9 + i] = j1[i];
    }
  }
  if (Jp) {
    T jp[6];
    jp_from(pl, ct, jp);
#pragma unroll
    for (int i = 0; i < 6; ++i) Jp[6 * k + i] = jp[i];
  }
  if (w) {
    const int j = cm_pt[s];
    const T* X = pts_buf + (long long)st->cur * 3 * P + 3LL * j;
    T px, py, sc;
    project_obs(ct, X[0], X[1], X[2], px, py, sc);
    const T r0 = sc * px - cm_px[s], r1 = sc * py - cm_px[(long long)O + s];
    T hr, ww;
    huber_weight(r0 * r0 + r1 * r1, delta, hr, ww);
    w[k] = ww;
  }
}

}  // namespace ba
