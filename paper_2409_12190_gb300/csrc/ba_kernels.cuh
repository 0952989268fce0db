// Device kernels of the LM bundle-adjustment hot path (sm_103a).
//
// Per observation k the weighted residual Jacobian (Sec. III-C) is kept in a
// factored form:
//   A = sqrt(w) d pi / d X_cam      (2x3)
//   q = sqrt(w) (d, f |p|^2, f |p|^4)   so  d r / d(f, k1, k2) = p q^T  (2x3)
//   RX = R X                          (the rotated point)
// from which, with the camera's R and left Jacobian J_l,
//   camera block  Jc = [ A (-[RX]_x) J_l | A | p q^T ]   (2x9)
//   point block   Jp = A R                                (2x3).
// Products with Jc, Jc^T, Jp, Jp^T are applied in this factored form;
// W_k = Jc^T Jp is never formed.
//
// Two storage modes (a template flag MF on the kernels that need it):
//   stored  (MF = false)  the 24 numbers A, B = A (-[RX]_x) J_l, D = p q^T and
//            Jp = A R are written once per linearisation, in camera-major
//            order, as structure-of-arrays planes of length O, and every later
//            pass streams them (the FP64 path: FP64 arithmetic is scarce on
//            this GPU, bytes are not; storing Jp saves the passes the 15 FMAs
//            of forming A^T e and R^T (.) or R t and A (.) per observation);
//   recompute (MF = true) nothing per observation but sqrt(w) (only under a
//            robust loss) is stored; every pass recomputes A, q, RX from the
//            point, the camera table and sqrt(w) (the FP32 path: ~60 FP32
//            operations per observation replace ~72 bytes of HBM traffic).
//
// Per-camera tables (T = float or double):
//   camtab [C][32]: R[0..8] t[9..11] f k1 k2 [12..14] pad, J_l[16..24], pad
//   a PCG vector x in factored form [C][12]: J_l x_omega, x_t, x_i, pad, so
//   that Jc x = A (u x RX + x_t) + p (q . x_i).
// Per camera U [45] (packed upper triangle), gc [9], block-Jacobi inverse
// [45]; per point V [6], gp [3], V*^{-1} [6], y0 = V*^{-1} gp [3] (double for
// the sums, T for what the passes read) and a 32-byte-aligned record
// ptab [P][8] = (X, 0, t, 0) holding the point and the PCG point vector, so
// that each per-observation point access is one vector load.
//
// The implicit Schur product S p = U* p - W V*^{-1} W^T p runs as three
// passes, the two heavy ones camera-major (the camera's data in registers):
//   A1 (camera-major)  z_k = Jp_k^T Jc_k p_c            -> one 4-vector per obs
//   A2 (point-major)   t_j = V*_j^{-1} sum_{k in j} z_k   (gather through the
//                      point-to-camera order map, segmented sum per point;
//                      with the points renumbered by first camera the
//                      gathers are nearly sequential)
//   B  (camera-major)  sum_{k in c} Jc_k^T Jp_k t_p(k)   -> per-piece partials
//
// Reductions.  Every sum over observations is taken in a fixed order: a
// camera's observations are cut into pieces of at most PIECE slots, one CTA
// per piece reduces its slots (per-thread partials, warp shuffles, then the
// warps in order) and a per-camera kernel adds the pieces in order; points
// are grouped into chunks of at most CHUNK_SLOTS observations, one CTA per
// chunk computes one observation per thread into shared memory and one
// thread per point adds its observations in slot order.  No global atomics
// are used on the numeric path, so every result is bitwise reproducible.
// Per-observation arithmetic and per-thread partial sums are in T; sums
// across warps, dot products, costs and the gain ratio are in double.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ba.h"

namespace ba {

constexpr int PIECE = 2048;          // max camera-major slots per piece
constexpr int PIECE_THREADS = 256;
constexpr int PASSB_THREADS = 128;    // pass B and the cost pass, FP32 recompute mode
// The linearisation and Schur-block passes reduce 54 values per piece in
// float-float arithmetic; fewer threads per piece spread that reduction over
// more slots per thread.
constexpr int LIN_THREADS = 64;
constexpr int PT_THREADS = 256;
constexpr int CAM_THREADS = 32;
constexpr int NPLANE = 24;     // stored planes: A (6), B (6), D (6), Jp = A R (6)
constexpr int NPLANE_JC = 18;  // the first 18: the camera block Jc = [B | A | D]
constexpr int CT = 32;               // camera table stride
constexpr int CT_T = 9, CT_F = 12, CT_K1 = 13, CT_K2 = 14, CT_JL = 16;
constexpr int PV = 12;               // factored PCG vector stride
constexpr int PART = 64;             // doubles per piece partial (54 used)
constexpr int CHUNK_SLOTS = 1024;    // max point-major slots per point chunk
constexpr int CHUNK_PTS = 512;       // max points per point chunk
constexpr int CHUNK_THREADS = 256;
// fused pass A: staged cameras per chunk, padded row strides (different
// cameras in different banks)
constexpr int FA_CAMS = 128;
constexpr int FA_CT = 17;  // padded strides: different cameras in different banks
constexpr int FA_XV = 13;
// dynamic shared memory of k_pass_fa: z per slot, the chunk's points, then
// the tables and vectors of at most nc cameras (the most any chunk sees)
template <typename T>
constexpr int fa_smem(int nc) {
  return ((CHUNK_SLOTS + CHUNK_PTS) * 4 + nc * (FA_CT + FA_XV)) * (int)sizeof(T);
}
// dynamic shared memory of k_lin_pt: its per-slot sums, and with the chunk
// headers the chunk's camera tables and points
template <typename T>
constexpr int lin_pt_smem(bool staged) {
  return (CHUNK_SLOTS * 9 + (staged ? FA_CAMS * FA_CT + CHUNK_PTS * 3 : 0)) * (int)sizeof(T);
}

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
  int need_cost;     // F is stale (parameters or pixels replaced since)
};

__host__ __device__ constexpr int sym9(int i, int j) { return 9 * i - (i * (i - 1)) / 2 + (j - i); }
__host__ __device__ constexpr int sym3(int i, int j) { return 3 * i - (i * (i - 1)) / 2 + (j - i); }

template <typename V>
__device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Error-free sum of two floats: s + e == a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// (hi, lo) += (h2, l2) in float-float arithmetic (about 48 significant bits).
__device__ __forceinline__ void ff_add(float& hi, float& lo, float h2, float l2) {
  float s, e;
  two_sum(hi, h2, s, e);
  e += lo + l2;
  hi = s + e;
  lo = e - (hi - s);
}

// Float-float products (Dekker's product with the exact FMA remainder):
// (hi, lo) = (ah, al) * (bh, bl), and the same with a plain float b.
__device__ __forceinline__ void ff_mul(float ah, float al, float bh, float bl, float& hi, float& lo) {
  const float p = ah * bh;
  const float e = fmaf(ah, bh, -p) + (ah * bl + al * bh);
  hi = p + e;
  lo = e - (hi - p);
}
__device__ __forceinline__ void ff_mulf(float ah, float al, float b, float& hi, float& lo) {
  const float p = ah * b;
  const float e = fmaf(ah, b, -p) + al * b;
  hi = p + e;
  lo = e - (hi - p);
}
// (hi, lo) = 1 / (bh, bl): a reciprocal and one Newton correction.
__device__ __forceinline__ void ff_rcp(float bh, float bl, float& hi, float& lo) {
  const float q = 1.0f / bh;
  const float r = fmaf(-bh, q, 1.0f) - bl * q;  // 1 - b q, to first order
  const float c = r * q;
  hi = q + c;
  lo = c - (hi - q);
}

// Warp reduce-scatter of 64 float-float values: five shuffle steps, each
// halving the values a lane keeps (its partner lane takes the other half),
// 62 shuffled pairs in all instead of 5 x 64.  Lane l returns the warp totals
// of values 2l and 2l + 1 (after the step of offset o a lane keeps the upper
// half iff its lane bit o is set, so the kept block starts at 2l).  The order
// of the additions depends on the lane numbers only.
template <int N, int OFF>
__device__ __forceinline__ void rs_ff_step(float (&h)[32], float (&l)[32], int lane) {
  const bool up = (lane & OFF) != 0;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float kh = up ? h[N + i] : h[i], kl = up ? l[N + i] : l[i];
    const float gh = up ? h[i] : h[N + i], gl = up ? l[i] : l[N + i];
    const float rh = __shfl_xor_sync(0xffffffffu, gh, OFF), rl = __shfl_xor_sync(0xffffffffu, gl, OFF);
    ff_add(kh, kl, rh, rl);
    h[i] = kh;
    l[i] = kl;
  }
}
// The same reduce-scatter for 16 plain floats (four steps, 15 shuffles):
// lane l returns the warp total of value l >> 1 (lanes 2m and 2m + 1 both
// hold value m).
template <int N, int OFF>
__device__ __forceinline__ void rs_f_step(float (&h)[16], int lane) {
  const bool up = (lane & OFF) != 0;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const float k = up ? h[N + i] : h[i];
    const float g = up ? h[i] : h[N + i];
    h[i] = k + __shfl_xor_sync(0xffffffffu, g, OFF);
  }
}
__device__ __forceinline__ float warp_rs16_f(const float (&v)[16]) {
  const int lane = threadIdx.x & 31;
  float h[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) h[i] = v[i];
  rs_f_step<8, 16>(h, lane);
  rs_f_step<4, 8>(h, lane);
  rs_f_step<2, 4>(h, lane);
  rs_f_step<1, 2>(h, lane);
  return h[0] + __shfl_xor_sync(0xffffffffu, h[0], 1);
}

__device__ __forceinline__ void warp_rs64_ff(const float (&v)[64], float& h0, float& l0, float& h1, float& l1) {
  const int lane = threadIdx.x & 31;
  float h[32], l[32];
  const bool up = (lane & 16) != 0;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const float keep = up ? v[32 + i] : v[i];
    const float give = up ? v[i] : v[32 + i];
    two_sum(keep, __shfl_xor_sync(0xffffffffu, give, 16), h[i], l[i]);
  }
  rs_ff_step<16, 8>(h, l, lane);
  rs_ff_step<8, 4>(h, l, lane);
  rs_ff_step<4, 2>(h, l, lane);
  rs_ff_step<2, 1>(h, l, lane);
  h0 = h[0];
  l0 = l[0];
  h1 = h[1];
  l1 = l[1];
}

// Sum NV per-thread values over the block and write them to out (NV
// doubles), warps then the warps in order.  Doubles are reduced in double.
// blockDim.x <= 1024.
// Floats are reduced in float-float (PRECISE) -- as accurate as a double
// reduction of the float partials but on the FP32 pipes, which on this GPU
// are 64x faster than FP64 -- or in plain float for PCG products.  All
// threads must call it.
template <int NV, bool PRECISE = true>
__device__ __forceinline__ void block_sum_store(double (&v)[NV], double* __restrict__ out) {
  __shared__ double red[32][NV];
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

template <int NV, bool PRECISE = true>
__device__ __forceinline__ void block_sum_store(float (&v)[NV], double* __restrict__ out) {
  __shared__ float2 redf[32][NV];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  if constexpr (PRECISE && NV > 32 && NV <= 64) {
    float w[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) w[i] = i < NV ? v[i] : 0.f;
    float h0, l0, h1, l1;
    warp_rs64_ff(w, h0, l0, h1, l1);
    if (2 * lane < NV) redf[warp][2 * lane] = make_float2(h0, l0);
    if (2 * lane + 1 < NV) redf[warp][2 * lane + 1] = make_float2(h1, l1);
  } else if constexpr (!PRECISE && NV > 4 && NV <= 16) {
    float w[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) w[i] = i < NV ? v[i] : 0.f;
    const float s = warp_rs16_f(w);
    if ((lane & 1) == 0 && (lane >> 1) < NV) redf[warp][lane >> 1] = make_float2(s, 0.f);
  } else {
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    float hi = v[i], lo = 0.f;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float h2 = __shfl_xor_sync(0xffffffffu, hi, off);
      if (PRECISE) {
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, off);
        ff_add(hi, lo, h2, l2);
      } else {
        hi += h2;
      }
    }
    if (lane == 0) redf[warp][i] = make_float2(hi, lo);
  }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NV; i += blockDim.x) {
    float hi = redf[0][i].x, lo = redf[0][i].y;
    for (int w = 1; w < nw; ++w) {
      if (PRECISE) ff_add(hi, lo, redf[w][i].x, redf[w][i].y);
      else hi += redf[w][i].x;
    }
    out[i] = (double)hi + (double)lo;
  }
}

// Block sum of NV doubles, returned to every thread.
template <int NV>
__device__ __forceinline__ void block_sum_all(double (&v)[NV]) {
  __shared__ double red2[32][NV];
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

// Fixed-order sum of n doubles (a[i * stride]) by the whole block; every
// thread gets the total.
__device__ __forceinline__ double block_sum_array(const double* __restrict__ a, int n, int stride) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += a[(long long)i * stride];
  double v[1] = {s};
  block_sum_all<1>(v);
  return v[0];
}

// Fixed-order sums of N arrays of n doubles at once (one block reduction).
template <int N>
__device__ __forceinline__ void block_sum_arrays(const double* const (&a)[N], int n, double (&out)[N]) {
#pragma unroll
  for (int k = 0; k < N; ++k) out[k] = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
#pragma unroll
    for (int k = 0; k < N; ++k) out[k] += a[k][i];
  block_sum_all<N>(out);
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
    ct[CT_JL + i] = (T)Jl[i];
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) ct[CT_T + i] = cam[3 + i];
  ct[15] = T(0);
#pragma unroll
  for (int i = 25; i < CT; ++i) ct[i] = T(0);
}

// The camera table in double from parameters of either precision (the FP32
// variant evaluates its cost in FP64: see cost_cam_range).
template <typename T>
__device__ inline void camera_table_f64(const T* __restrict__ cam, double* __restrict__ ct) {
  double R[9], Jl[9];
  so3_tables((double)cam[0], (double)cam[1], (double)cam[2], R, Jl);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    ct[i] = R[i];
    ct[CT_JL + i] = Jl[i];
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) ct[CT_T + i] = (double)cam[3 + i];
  ct[15] = 0.0;
#pragma unroll
  for (int i = 25; i < CT; ++i) ct[i] = 0.0;
}

// ---------------------------------------------------------------------------
// One observation
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ void project_obs(const T* __restrict__ ct, T X0, T X1, T X2,
                                            T& px, T& py, T& s) {
  const T P0 = ct[0] * X0 + ct[1] * X1 + ct[2] * X2 + ct[CT_T];
  const T P1 = ct[3] * X0 + ct[4] * X1 + ct[5] * X2 + ct[CT_T + 1];
  const T P2 = ct[6] * X0 + ct[7] * X1 + ct[8] * X2 + ct[CT_T + 2];
  const T iz = T(1) / P2;
  px = -P0 * iz;
  py = -P1 * iz;
  const T r2 = px * px + py * py;
  s = ct[CT_F] * (T(1) + r2 * (ct[CT_K1] + ct[CT_K2] * r2));
}

// A camera table (R, t, f, k1, k2: the first 15 entries of the double
// table) split into float-float pairs, for the FP32 variant's cost.
struct FFCam {
  float h[15], l[15];
};
__device__ __forceinline__ void ffcam_from(const double* __restrict__ ct, FFCam& o) {
#pragma unroll
  for (int i = 0; i < 15; ++i) {
    o.h[i] = (float)ct[i];
    o.l[i] = (float)(ct[i] - (double)o.h[i]);
  }
}

// Squared residual |pi(theta_c, X) - x|^2 in float-float arithmetic (about
// 44 significant bits after the division), returned as a double; X and the
// pixel are FP32 values (exact in float-float).  The projection of
// project_obs, step for step.
__device__ __forceinline__ double sq_residual_ff(const FFCam& c, float X0, float X1, float X2, float u0, float u1) {
  float Ph[3], Pl[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float h, l, h2, l2;
    ff_mulf(c.h[3 * a], c.l[3 * a], X0, h, l);
    ff_mulf(c.h[3 * a + 1], c.l[3 * a + 1], X1, h2, l2);
    ff_add(h, l, h2, l2);
    ff_mulf(c.h[3 * a + 2], c.l[3 * a + 2], X2, h2, l2);
    ff_add(h, l, h2, l2);
    ff_add(h, l, c.h[CT_T + a], c.l[CT_T + a]);
    Ph[a] = h;
    Pl[a] = l;
  }
  float izh, izl, pxh, pxl, pyh, pyl;
  ff_rcp(Ph[2], Pl[2], izh, izl);
  ff_mul(-Ph[0], -Pl[0], izh, izl, pxh, pxl);
  ff_mul(-Ph[1], -Pl[1], izh, izl, pyh, pyl);
  float r2h, r2l, th, tl;
  ff_mul(pxh, pxl, pxh, pxl, r2h, r2l);
  ff_mul(pyh, pyl, pyh, pyl, th, tl);
  ff_add(r2h, r2l, th, tl);
  // s = f (1 + r2 (k1 + k2 r2))
  float dh, dl;
  ff_mul(c.h[CT_K2], c.l[CT_K2], r2h, r2l, dh, dl);
  ff_add(dh, dl, c.h[CT_K1], c.l[CT_K1]);
  ff_mul(dh, dl, r2h, r2l, th, tl);
  ff_add(th, tl, 1.0f, 0.0f);
  float sh, sl;
  ff_mul(c.h[CT_F], c.l[CT_F], th, tl, sh, sl);
  float r0h, r0l, r1h, r1l;
  ff_mul(sh, sl, pxh, pxl, r0h, r0l);
  ff_mul(sh, sl, pyh, pyl, r1h, r1l);
  ff_add(r0h, r0l, -u0, 0.0f);
  ff_add(r1h, r1l, -u1, 0.0f);
  float qh, ql;
  ff_mul(r0h, r0l, r0h, r0l, qh, ql);
  ff_mul(r1h, r1l, r1h, r1l, th, tl);
  ff_add(qh, ql, th, tl);
  return (double)qh + (double)ql;
}

// Huber on |r|: half_rho = 1/2 rho(s); returns sqrt(w), w = rho'(s).
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

// Factored Jacobian of one observation (weights folded in).
template <typename T>
struct Fac {
  T RX0, RX1, RX2;   // R X
  T px, py;          // normalised image point
  T A[6];            // sqrt(w) d pi / d X_cam
  T q0, q1, q2;      // sqrt(w) (d, f |p|^2, f |p|^4)
};

// d pi / d p = s I + m p p^T (s = f d, m = f (2 k1 + 4 k2 |p|^2));
// d p / d X_cam = -(1/X_cam[2]) [[1, 0, p_x], [0, 1, p_y]].
template <typename T>
__device__ __forceinline__ void fac_obs(const T* __restrict__ ct, T X0, T X1, T X2, T sw, Fac<T>& o) {
  o.RX0 = ct[0] * X0 + ct[1] * X1 + ct[2] * X2;
  o.RX1 = ct[3] * X0 + ct[4] * X1 + ct[5] * X2;
  o.RX2 = ct[6] * X0 + ct[7] * X1 + ct[8] * X2;
  const T P0 = o.RX0 + ct[CT_T], P1 = o.RX1 + ct[CT_T + 1], P2 = o.RX2 + ct[CT_T + 2];
  const T f = ct[CT_F], k1 = ct[CT_K1], k2 = ct[CT_K2];
  const T iz = T(1) / P2;
  const T px = -P0 * iz, py = -P1 * iz;
  o.px = px;
  o.py = py;
  const T r2 = px * px + py * py;
  const T d = T(1) + r2 * (k1 + k2 * r2);
  const T s = f * d;
  const T m = f * (T(2) * k1 + T(4) * k2 * r2);
  const T a00 = s + m * px * px, a01 = m * px * py, a11 = s + m * py * py;
  const T n = -iz * sw;
  o.A[0] = n * a00;
  o.A[1] = n * a01;
  o.A[2] = n * (a00 * px + a01 * py);
  o.A[3] = n * a01;
  o.A[4] = n * a11;
  o.A[5] = n * (a01 * px + a11 * py);
  o.q0 = sw * d;
  o.q1 = sw * f * r2;
  o.q2 = o.q1 * r2;
}

template <typename T>
__device__ __forceinline__ void jp_from(const T* __restrict__ A, const T* __restrict__ R, T (&Jp)[6]);

// Planes A, B = A (-[RX]_x) J_l, D = p q^T and the point block Jp = A R from
// the factored form (ct: the camera table, R at 0 and J_l at CT_JL).
template <typename T>
__device__ __forceinline__ void fac_planes(const Fac<T>& o, const T* __restrict__ ct, T (&pl)[NPLANE]) {
  const T* Jl = ct + CT_JL;
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const T* Ar = o.A + 3 * a;
    // row a of A (-[RX]_x) = RX x A_row, then times J_l
    const T c0 = o.RX1 * Ar[2] - o.RX2 * Ar[1];
    const T c1 = o.RX2 * Ar[0] - o.RX0 * Ar[2];
    const T c2 = o.RX0 * Ar[1] - o.RX1 * Ar[0];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      pl[3 * a + j] = Ar[j];
      pl[6 + 3 * a + j] = c0 * Jl[j] + c1 * Jl[3 + j] + c2 * Jl[6 + j];
    }
    const T pa = a == 0 ? o.px : o.py;
    pl[12 + 3 * a] = pa * o.q0;
    pl[13 + 3 * a] = pa * o.q1;
    pl[14 + 3 * a] = pa * o.q2;
  }
  T jp[6];
  jp_from(o.A, ct, jp);
#pragma unroll
  for (int i = 0; i < 6; ++i) pl[NPLANE_JC + i] = jp[i];
}

// Residual, weight and factored Jacobian of one observation.
template <typename T>
__device__ __forceinline__ void lin_obs(const T* __restrict__ ct, T X0, T X1, T X2, T u0, T u1, T delta,
                                        Fac<T>& o, T& r0w, T& r1w, T& half_rho, T& sw) {
  T px, py, s;
  project_obs(ct, X0, X1, X2, px, py, s);
  const T r0 = s * px - u0, r1 = s * py - u1;
  T w;
  sw = huber_weight(r0 * r0 + r1 * r1, delta, half_rho, w);
  r0w = sw * r0;
  r1w = sw * r1;
  fac_obs(ct, X0, X1, X2, sw, o);
}

// Camera rows of Jc = [B | A | D] as 9 values each.
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

// The stored planes are interleaved in pairs: plane p of slot s is
// J[((p / 2) O + s) 2 + p % 2], so a thread reads two planes with one
// 2-vector load and a warp still reads contiguous memory.
template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
  using type = float2;
};
template <>
struct Vec2<double> {
  using type = double2;
};

// The first N planes (N even) of camera-major slot s (N = NPLANE_JC when Jp
// is not needed).
template <int N = NPLANE, typename T>
__device__ __forceinline__ void load_planes(const T* __restrict__ J, long long O, long long s, T (&pl)[NPLANE]) {
  static_assert(N % 2 == 0, "planes are read in pairs");
  using V2 = typename Vec2<T>::type;
#pragma unroll
  for (int q = 0; q < N / 2; ++q) {
    const V2 v = reinterpret_cast<const V2*>(J)[(long long)q * O + s];
    pl[2 * q] = v.x;
    pl[2 * q + 1] = v.y;
  }
}

// Four consecutive T as one vector access (the address is 4 * sizeof(T)
// aligned: every caller indexes a stride-4 or stride-8 table).
__device__ __forceinline__ void load4(const float* __restrict__ p, float& a, float& b, float& c, float& d) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = v.x; b = v.y; c = v.z; d = v.w;
}
__device__ __forceinline__ void load4(const double* __restrict__ p, double& a, double& b, double& c, double& d) {
  const double2 v0 = reinterpret_cast<const double2*>(p)[0];
  const double2 v1 = reinterpret_cast<const double2*>(p)[1];
  a = v0.x; b = v0.y; c = v1.x; d = v1.y;
}
__device__ __forceinline__ void store4(float* __restrict__ p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void store4(double* __restrict__ p, double a, double b, double c, double d) {
  reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
  reinterpret_cast<double2*>(p)[1] = make_double2(c, d);
}

// Jc x with x in factored form xv = [J_l x_omega, x_t, x_i].
template <typename T>
__device__ __forceinline__ void jc_times_fac(const Fac<T>& o, const T* __restrict__ xv, T& e0, T& e1) {
  const T w0 = xv[1] * o.RX2 - xv[2] * o.RX1 + xv[3];
  const T w1 = xv[2] * o.RX0 - xv[0] * o.RX2 + xv[4];
  const T w2 = xv[0] * o.RX1 - xv[1] * o.RX0 + xv[5];
  const T qi = o.q0 * xv[6] + o.q1 * xv[7] + o.q2 * xv[8];
  e0 = o.A[0] * w0 + o.A[1] * w1 + o.A[2] * w2 + o.px * qi;
  e1 = o.A[3] * w0 + o.A[4] * w1 + o.A[5] * w2 + o.py * qi;
}

// Jc^T h accumulated in the form [RX x (A^T h) | A^T h | q (p . h)]: the
// first three must still be multiplied by J_l^T (per camera, once per sum).
template <typename T>
__device__ __forceinline__ void jct_fac_acc(const Fac<T>& o, T h0, T h1, T (&acc)[9]) {
  const T v0 = o.A[0] * h0 + o.A[3] * h1;
  const T v1 = o.A[1] * h0 + o.A[4] * h1;
  const T v2 = o.A[2] * h0 + o.A[5] * h1;
  acc[0] += o.RX1 * v2 - o.RX2 * v1;
  acc[1] += o.RX2 * v0 - o.RX0 * v2;
  acc[2] += o.RX0 * v1 - o.RX1 * v0;
  acc[3] += v0;
  acc[4] += v1;
  acc[5] += v2;
  const T ph = o.px * h0 + o.py * h1;
  acc[6] += o.q0 * ph;
  acc[7] += o.q1 * ph;
  acc[8] += o.q2 * ph;
}

// Factored form of a camera vector x: [J_l x_omega, x_t, x_i, 0, 0, 0].
template <typename T>
__device__ __forceinline__ void to_factored(const T* __restrict__ Jl, const double* __restrict__ x,
                                            T* __restrict__ out) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
    out[i] = (T)((double)Jl[3 * i] * x[0] + (double)Jl[3 * i + 1] * x[1] + (double)Jl[3 * i + 2] * x[2]);
#pragma unroll
  for (int i = 3; i < 9; ++i) out[i] = (T)x[i];
  out[9] = out[10] = out[11] = T(0);
}

// ---------------------------------------------------------------------------
// Set-up kernels
// ---------------------------------------------------------------------------

template <typename T>
static __global__ void k_validate(int C, int P, int O, const T* __restrict__ cams, const T* __restrict__ pts,
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
static __global__ void k_gather_obs(int O, const int32_t* __restrict__ perm_cam, const int32_t* __restrict__ perm_pt,
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
static __global__ void k_project(int O, const T* __restrict__ cams, const T* __restrict__ pts,
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
static __global__ void k_cam_prep(int C, const T* __restrict__ cams_buf, const DevState* __restrict__ st,
                           int gate, T* __restrict__ camtab) {
  if (gate && !st->need_lin) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  camera_table(cams_buf + (long long)st->cur * 9 * C + 9LL * c, camtab + (long long)CT * c);
}

// Point table [P][8]: X in 0..2 (from the current parameters); 4..6 hold the
// PCG vector t that pass A writes for pass B.
template <typename T>
static __global__ void k_pt_prep(int P, const T* __restrict__ pts_buf, const DevState* __restrict__ st, int gate,
                          T* __restrict__ ptab) {
  if (gate && !st->need_lin) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P) return;
  const T* X = pts_buf + (long long)st->cur * 3 * P + 3LL * j;
  store4(ptab + 8LL * j, X[0], X[1], X[2], T(0));
}

// key_j = smallest camera that observes point j (C if none), from the
// stable CSR of the observations by point.
static __global__ void k_point_key(int P, int C, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ perm,
                            const int32_t* __restrict__ cam_idx, int32_t* __restrict__ key) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P) return;
  int k = C;
  for (int q = rowptr[j]; q < rowptr[j + 1]; ++q) k = min(k, cam_idx[perm[q]]);
  key[j] = k;
}

// dst[i] = src[idx[i]]
static __global__ void k_gather_i32(int n, const int32_t* __restrict__ idx, const int32_t* __restrict__ src,
                             int32_t* __restrict__ dst) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
}

// dst[i][:] = src[idx[i]][:] for rows of W values
// One int of the device state (stream-ordered, no host round trip).
static __global__ void k_set_int(int* p, int v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *p = v;
}

// Parameters in and out of the current buffer of the double-buffered
// parameter arrays, the buffer index read on the device: cameras [C][9] are
// copied, points [P][3] are gathered between the caller's numbering (rows
// of tmp) and the internal one (idx: internal -> caller row for the load,
// caller -> internal row for the store).
template <typename T>
static __global__ void k_cams_cur(long long n, const DevState* __restrict__ st, const T* __restrict__ src,
                                  T* __restrict__ cams, int store) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T* buf = cams + (long long)st->cur * n;
  if (store) buf[i] = src[i];
  else const_cast<T*>(src)[i] = buf[i];
}
template <typename T>
static __global__ void k_points_cur(int P, const int32_t* __restrict__ idx, const DevState* __restrict__ st,
                                    T* __restrict__ tmp, T* __restrict__ pts, int store) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  T* buf = pts + (long long)st->cur * 3 * P;
  const long long r = idx[i];
#pragma unroll
  for (int w = 0; w < 3; ++w) {
    if (store) buf[3 * i + w] = tmp[3 * r + w];
    else tmp[3 * i + w] = buf[3 * r + w];
  }
}

template <typename X, int W>
static __global__ void k_gather_rows(int n, const int32_t* __restrict__ idx, const X* __restrict__ src,
                              X* __restrict__ dst) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long r = idx[i];
#pragma unroll
  for (int w = 0; w < W; ++w) dst[W * i + w] = src[W * r + w];
}

// inv[perm[s]] = s
static __global__ void k_invert_perm(int O, const int32_t* __restrict__ perm, int32_t* __restrict__ inv) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < O) inv[perm[s]] = (int32_t)s;
}

// out[s] = inv_b[perm_a[s]]: the slot, in order b, of the observation at slot
// s of order a (e.g. the point-major slot of each camera-major slot).
static __global__ void k_compose_perm(int O, const int32_t* __restrict__ perm_a, const int32_t* __restrict__ inv_b,
                               int32_t* __restrict__ out) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < O) out[s] = inv_b[perm_a[s]];
}

// Camera-major slots [beg, end) of one camera, NT threads striding: residuals,
// weights and the per-thread partial U (45) and gc (9); in the stored mode
// also the planes, in any mode sqrt(w) when sw_out is given.
template <typename T, bool STORE, int NT>
__device__ __forceinline__ void lin_cam_range(int beg, int end, const int32_t* __restrict__ cm_pt,
                                              const T* __restrict__ cm_px, const T* __restrict__ pts,
                                              const T* __restrict__ sct, T delta, int O, T* __restrict__ Jcm,
                                              T* __restrict__ sw_out, T (&acc)[54]) {
  for (int s = beg + threadIdx.x; s < end; s += NT) {
    const int j = cm_pt[s];
    Fac<T> o;
    T r0, r1, hr, sw;
    lin_obs(sct, pts[3LL * j], pts[3LL * j + 1], pts[3LL * j + 2], cm_px[s], cm_px[(long long)O + s], delta, o,
            r0, r1, hr, sw);
    if (sw_out) sw_out[s] = sw;
    T pl[NPLANE];
    fac_planes(o, sct, pl);
    if (STORE) {
      using V2 = typename Vec2<T>::type;
#pragma unroll
      for (int q = 0; q < NPLANE / 2; ++q) {
        V2 v;
        v.x = pl[2 * q];
        v.y = pl[2 * q + 1];
        reinterpret_cast<V2*>(Jcm)[(long long)q * O + s] = v;
      }
    }
    T j0[9], j1[9];
    jc_rows(pl, j0, j1);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
#pragma unroll
      for (int k = i; k < 9; ++k) acc[sym9(i, k)] += j0[i] * j0[k] + j1[i] * j1[k];
      acc[45 + i] += j0[i] * r0 + j1[i] * r1;
    }
  }
}

// Camera-major pass: residuals, weights, U (45) and gc (9) per piece; in the
// stored mode also the planes, in any mode sqrt(w) when sw_out is given.
template <typename T, bool STORE>
static __global__ void __launch_bounds__(LIN_THREADS)
k_lin_cam(const int32_t* __restrict__ piece_cam, const int32_t* __restrict__ piece_beg,
          const int32_t* __restrict__ piece_end, const int32_t* __restrict__ cm_pt,
          const T* __restrict__ cm_px, const T* __restrict__ pts_buf, const T* __restrict__ camtab,
          const DevState* __restrict__ st, int gate, T delta, int O, int P, T* __restrict__ Jcm,
          T* __restrict__ sw_out, double* __restrict__ part) {
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
  lin_cam_range<T, STORE, LIN_THREADS>(piece_beg[b], piece_end[b], cm_pt, cm_px, pts, sct, delta, O, Jcm, sw_out,
                                         acc);
  block_sum_store<54>(acc, part + (long long)PART * b);
}

// Add pieces [p0, p1) of one camera in order: U (45), gc (9).
__device__ __forceinline__ void cam_combine_lin_one(int p0, int p1, const double* __restrict__ part,
                                                    double* __restrict__ U, double* __restrict__ gc) {
  for (int i = 0; i < 54; ++i) {
    double s = 0.0;
    for (int p = p0; p < p1; ++p) s += part[(long long)PART * p + i];
    if (i < 45) U[i] = s;
    else gc[i - 45] = s;
  }
}

// Add the pieces of each camera in order: U [C][45], gc [C][9].
static __global__ void k_cam_combine_lin(int C, const int32_t* __restrict__ cam_piece_ptr,
                                  const double* __restrict__ part, const DevState* __restrict__ st,
                                  int gate, double* __restrict__ U, double* __restrict__ gc) {
  if (gate && !st->need_lin) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  cam_combine_lin_one(cam_piece_ptr[c], cam_piece_ptr[c + 1], part, U + 45LL * c, gc + 9LL * c);
}

// Point-major pass over one chunk of points: V (6) and gp (3) per point,
// and sqrt(w) when sw_out is given.  One thread per observation (coalesced);
// each observation's 9 contributions go to shared memory and one thread per
// point adds its observations in slot order.  A point with more than
// CHUNK_SLOTS observations is a chunk of its own and is reduced by the block.
template <typename T>
__device__ __forceinline__ void lin_pt_obs(int q, int O, const int32_t* __restrict__ pm_cam,
                                           const int32_t* __restrict__ pm_pt, const T* __restrict__ pm_px,
                                           const T* __restrict__ pts, const T* __restrict__ camtab, T delta,
                                           T* __restrict__ sw_out, T (&v)[9]) {
  const int j = pm_pt[q];
  const T* ct = camtab + (long long)CT * pm_cam[q];
  T ctl[CT];
#pragma unroll
  for (int i = 0; i < CT; ++i) ctl[i] = ct[i];
  Fac<T> o;
  T r0, r1, hr, sw;
  lin_obs(ctl, pts[3LL * j], pts[3LL * j + 1], pts[3LL * j + 2], pm_px[q], pm_px[(long long)O + q], delta, o, r0,
          r1, hr, sw);
  if (sw_out) sw_out[q] = sw;
  T Jp[6];
  jp_from(o.A, ctl, Jp);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = a; b < 3; ++b) v[sym3(a, b)] = Jp[a] * Jp[b] + Jp[3 + a] * Jp[3 + b];
    v[6 + a] = Jp[a] * r0 + Jp[3 + a] * r1;
  }
}

// lin_pt_obs with the camera table ct and the point X from shared memory.
template <typename T>
__device__ __forceinline__ void lin_pt_obs_staged(int q, int O, const T* __restrict__ pm_px, const T* ct, T X0, T X1,
                                                  T X2, T delta, T* __restrict__ sw_out, T (&v)[9]) {
  Fac<T> o;
  T r0, r1, hr, sw;
  lin_obs(ct, X0, X1, X2, pm_px[q], pm_px[(long long)O + q], delta, o, r0, r1, hr, sw);
  if (sw_out) sw_out[q] = sw;
  T Jp[6];
  jp_from(o.A, ct, Jp);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = a; b < 3; ++b) v[sym3(a, b)] = Jp[a] * Jp[b] + Jp[3 + a] * Jp[3 + b];
    v[6 + a] = Jp[a] * r0 + Jp[3 + a] * r1;
  }
}

template <typename T>
static __global__ void __launch_bounds__(CHUNK_THREADS)
k_lin_pt(const int32_t* __restrict__ pchunk, int O, const int32_t* __restrict__ rowptr_pt,
         const int32_t* __restrict__ pm_cam, const int32_t* __restrict__ pm_pt, const T* __restrict__ pm_px,
         const T* __restrict__ pts_buf, const T* __restrict__ camtab, const DevState* __restrict__ st, int P,
         int gate, T delta, T* __restrict__ sw_out, double* __restrict__ V, double* __restrict__ gp,
         const int4* __restrict__ chunk_hdr, const int16_t* __restrict__ pm_lc,
         const int32_t* __restrict__ chunk_cams) {
  if (gate && !st->need_lin) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sv = reinterpret_cast<T*>(smem_raw);  // [CHUNK_SLOTS][9]
  const T* pts = pts_buf + (long long)st->cur * 3 * P;
  const int j0 = pchunk[blockIdx.x], j1 = pchunk[blockIdx.x + 1];
  const int s0 = rowptr_pt[j0], s1 = rowptr_pt[j1];
  if (s1 - s0 <= CHUNK_SLOTS && chunk_hdr) {
    // with the fused pass's chunk headers: the chunk's camera tables and its
    // (consecutive) points staged in shared memory, as in k_pass_fa
    T* sct = sv + CHUNK_SLOTS * 9;  // [FA_CAMS][FA_CT]
    T* sX = sct + FA_CAMS * FA_CT;   // [CHUNK_PTS][3]
    const int4 h1 = chunk_hdr[2 * blockIdx.x + 1];
    const int c0 = h1.x, nc = h1.y, cmin = h1.z;
    for (int i = threadIdx.x; i < nc * 16; i += CHUNK_THREADS) {
      const int l = i >> 4, e = i & 15;
      const int cam = cmin >= 0 ? cmin + l : chunk_cams[c0 + l];
      if (e < 15) sct[l * FA_CT + e] = camtab[(long long)CT * cam + e];
    }
    for (int i = threadIdx.x; i < 3 * (j1 - j0); i += CHUNK_THREADS) sX[i] = pts[3LL * j0 + i];
    __syncthreads();
    for (int q = s0 + threadIdx.x; q < s1; q += CHUNK_THREADS) {
      const int jl = pm_pt[q] - j0;
      T v[9];
      lin_pt_obs_staged<T>(q, O, pm_px, sct + pm_lc[q] * FA_CT, sX[3 * jl], sX[3 * jl + 1], sX[3 * jl + 2], delta,
                           sw_out, v);
#pragma unroll
      for (int i = 0; i < 9; ++i) sv[(q - s0) * 9 + i] = v[i];
    }
    __syncthreads();
  } else if (s1 - s0 <= CHUNK_SLOTS) {
    for (int q = s0 + threadIdx.x; q < s1; q += CHUNK_THREADS) {
      T v[9];
      lin_pt_obs<T>(q, O, pm_cam, pm_pt, pm_px, pts, camtab, delta, sw_out, v);
#pragma unroll
      for (int i = 0; i < 9; ++i) sv[(q - s0) * 9 + i] = v[i];
    }
    __syncthreads();
  }
  if (s1 - s0 <= CHUNK_SLOTS) {
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
      lin_pt_obs<T>(q, O, pm_cam, pm_pt, pm_px, pts, camtab, delta, sw_out, v);
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
__device__ __forceinline__ void pt_damp_one(int j, const double* __restrict__ V, const double* __restrict__ gp,
                                            double lam, double dmin, double dmax, T* __restrict__ Vinv,
                                            T* __restrict__ y0) {
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

template <typename T>
static __global__ void k_pt_damp(int P, const double* __restrict__ V, const double* __restrict__ gp,
                          const double* __restrict__ lam_ptr, double dmin, double dmax,
                          T* __restrict__ Vinv, T* __restrict__ y0) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P) return;
  pt_damp_one<T>(j, V, gp, *lam_ptr, dmin, dmax, Vinv, y0);
}

// The planes of camera-major slot s: loaded (stored mode) or recomputed.
template <typename T, bool MF>
__device__ __forceinline__ void cm_planes(const T* __restrict__ Jcm, long long O, int s, const T* __restrict__ sct,
                                          const T* __restrict__ pts, int j, const T* __restrict__ sw,
                                          T (&pl)[NPLANE]) {
  if (MF) {
    Fac<T> o;
    fac_obs(sct, pts[3LL * j], pts[3LL * j + 1], pts[3LL * j + 2], sw ? sw[s] : T(1), o);
    fac_planes(o, sct, pl);
  } else {
    load_planes(Jcm, O, s, pl);
  }
}

// Camera-major slots [beg, end), NT threads striding: per-thread partial
// sum_k Jc^T (Jp V*^{-1} Jp^T) Jc (45) and sum_k Jc^T Jp y0 (9).
template <typename T, bool MF, int NT>
__device__ __forceinline__ void schur_cam_range(int beg, int end, const int32_t* __restrict__ cm_pt,
                                                const T* __restrict__ Jcm, const T* __restrict__ sct,
                                                const T* __restrict__ pts, const T* __restrict__ cm_sw,
                                                const T* __restrict__ Vinv, const T* __restrict__ y0, int O,
                                                T (&acc)[54]) {
  for (int s = beg + threadIdx.x; s < end; s += NT) {
    const int j = cm_pt[s];
    T pl[NPLANE];
    cm_planes<T, MF>(Jcm, O, s, sct, pts, j, cm_sw, pl);
    const T* Jp = pl + NPLANE_JC;
    const T* vi = Vinv + 6LL * j;
    const T v00 = vi[0], v01 = vi[1], v02 = vi[2], v11 = vi[3], v12 = vi[4], v22 = vi[5];
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
}

// Camera-major pass: per piece, sum_k Jc^T (Jp V*^{-1} Jp^T) Jc (45) and
// sum_k Jc^T Jp y0 (9).
template <typename T, bool MF>
static __global__ void __launch_bounds__(LIN_THREADS)
k_schur_cam(const int32_t* __restrict__ piece_cam, const int32_t* __restrict__ piece_beg,
            const int32_t* __restrict__ piece_end, const int32_t* __restrict__ cm_pt,
            const T* __restrict__ Jcm, const T* __restrict__ camtab, const T* __restrict__ pts_buf,
            const T* __restrict__ cm_sw, const DevState* __restrict__ st, int P, const T* __restrict__ Vinv,
            const T* __restrict__ y0, int O, double* __restrict__ part) {
  __shared__ T sct[CT];
  const int b = blockIdx.x;
  const int c = piece_cam[b];
  if (threadIdx.x < CT) sct[threadIdx.x] = camtab[(long long)CT * c + threadIdx.x];
  __syncthreads();
  const T* pts = pts_buf + (long long)st->cur * 3 * P;
  T acc[54];
#pragma unroll
  for (int i = 0; i < 54; ++i) acc[i] = T(0);
  schur_cam_range<T, MF, LIN_THREADS>(piece_beg[b], piece_end[b], cm_pt, Jcm, sct, pts, cm_sw, Vinv, y0, O, acc);
  block_sum_store<54>(acc, part + (long long)PART * b);
}

// Cholesky of a packed symmetric 9x9 (upper triangle, sym9) and its inverse,
// in double.  Returns false if a pivot is not positive/finite.
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

// The same inverse with one 81-double work array W (for kernels that must
// keep few registers): the strict
// lower triangle holds L, the diagonal L_ii and then 1 / L_ii, the strict
// upper triangle the strict lower triangle of L^{-1} transposed.  Loops are
// kept rolled (few registers; the same operation order wherever it is
// inlined).  Returns false if a pivot is not positive/finite.
__device__ inline bool spd_inverse9_w(const double* __restrict__ S, double* __restrict__ Minv, double* __restrict__ W) {
#pragma unroll 1
  for (int j = 0; j < 9; ++j) {
    double d = S[sym9(j, j)];
#pragma unroll 1
    for (int k = 0; k < j; ++k) d -= W[9 * j + k] * W[9 * j + k];
    if (!(d > 0.0) || !isfinite(d)) return false;
    const double ljj = sqrt(d);
    W[9 * j + j] = ljj;
    const double il = 1.0 / ljj;
#pragma unroll 1
    for (int i = j + 1; i < 9; ++i) {
      double s = S[sym9(j, i)];
#pragma unroll 1
      for (int k = 0; k < j; ++k) s -= W[9 * i + k] * W[9 * j + k];
      W[9 * i + j] = s * il;
    }
  }
  // L^{-1} row by row: Li_ii = 1 / L_ii, Li_ij = -(sum_{k=j}^{i-1} L_ik Li_kj) Li_ii
#pragma unroll 1
  for (int i = 0; i < 9; ++i) {
    const double dii = 1.0 / W[9 * i + i];
    W[9 * i + i] = dii;
#pragma unroll 1
    for (int j = 0; j < i; ++j) {
      double s = 0.0;
#pragma unroll 1
      for (int k = j; k < i; ++k) s += W[9 * i + k] * W[9 * j + k];  // Li_kj: diagonal (k = j) or transposed
      W[9 * j + i] = -s * dii;
    }
  }
  // M_ij = sum_{k >= max(i, j)} Li_ki Li_kj
#pragma unroll 1
  for (int i = 0; i < 9; ++i)
#pragma unroll 1
    for (int j = i; j < 9; ++j) {
      double s = 0.0;
#pragma unroll 1
      for (int k = j; k < 9; ++k) s += W[9 * i + k] * W[9 * j + k];
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

// Write the camera vector x (double, 9) as the passes read it: plain in the
// stored mode, factored ([J_l x_omega, x_t, x_i]) in the recompute mode.
template <typename T, bool MF>
__device__ __forceinline__ void write_pass_vec(const T* __restrict__ ct, const double* __restrict__ x,
                                               T* __restrict__ out) {
  if (MF) {
    to_factored(ct + CT_JL, x, out);
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) out[i] = (T)x[i];
  }
}

__host__ __device__ constexpr int pass_vec_stride(bool mf) { return mf ? PV : 9; }

// One camera: S_ii = U*_i - (sum of its Schur pieces [p0, p1)), b_i = -gc_i +
// (their right-hand-side part), M_i = S_ii^{-1} (or the inverse diagonal of
// U* when S_ii is not SPD in this precision: *fallback = 1); PCG start x = 0,
// r = b, z = p = M r, p also in the passes' form; returns r.z and b.b.
template <typename T, bool MF, bool ROLLED = false>
__device__ __forceinline__ void cam_schur_one(int p0, int p1, const double* __restrict__ part,
                                              const double* __restrict__ Uc, const double* __restrict__ gcc,
                                              const T* __restrict__ ct, double lam, double dmin, double dmax,
                                              const uint8_t* __restrict__ fixed_c, double* __restrict__ Mc,
                                              double* __restrict__ xc, double* __restrict__ rc,
                                              double* __restrict__ zc, double* __restrict__ pc,
                                              T* __restrict__ pTc, double& rz, double& bb, int& fallback,
                                              double* __restrict__ S_out = nullptr) {
  double S[45], bv[9];
#pragma unroll
  for (int i = 0; i < 45; ++i) S[i] = Uc[i];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    S[sym9(i, i)] += damp(Uc[sym9(i, i)], lam, dmin, dmax);
    bv[i] = -gcc[i];
  }
  for (int q = p0; q < p1; ++q) {
    const double* pp = part + (long long)PART * q;
#pragma unroll
    for (int i = 0; i < 45; ++i) S[i] -= pp[i];
#pragma unroll
    for (int i = 0; i < 9; ++i) bv[i] += pp[45 + i];
  }
  if (fixed_c) {
    // frozen parameters: the system restricted to the free ones,
    // S -> m S m + (I - m), b -> m b
    bool fz[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      fz[i] = fixed_c[i] != 0;
      if (fz[i]) bv[i] = 0.0;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i)
#pragma unroll
      for (int j = i; j < 9; ++j)
        if (fz[i] || fz[j]) S[sym9(i, j)] = i == j ? 1.0 : 0.0;
  }
  if (S_out) {
#pragma unroll
    for (int i = 0; i < 45; ++i) S_out[i] = S[i];
  }
  double M[45];
  fallback = 0;
  bool spd;
  if (ROLLED) {
    double W[81];
    spd = spd_inverse9_w(S, M, W);
  } else {
    spd = spd_inverse9(S, M);
  }
  if (!spd) {
    // not SPD in this precision: fall back to the inverse diagonal of U*
#pragma unroll
    for (int i = 0; i < 45; ++i) M[i] = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const double d = Uc[sym9(i, i)] + damp(Uc[sym9(i, i)], lam, dmin, dmax);
      M[sym9(i, i)] = 1.0 / d;
    }
    fallback = 1;
  }
#pragma unroll
  for (int i = 0; i < 45; ++i) Mc[i] = M[i];
  double zz[9];
  sym9_matvec(M, bv, zz);
  rz = 0.0;
  bb = 0.0;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    xc[i] = 0.0;
    rc[i] = bv[i];
    zc[i] = zz[i];
    pc[i] = zz[i];
    rz += bv[i] * zz[i];
    bb += bv[i] * bv[i];
  }
  write_pass_vec<T, MF>(ct, zz, pTc);
}

// Per camera: S_ii, b_i, M_i = S_ii^{-1}; PCG start x = 0, r = b, z = M r,
// p = z; per-block partial sums of r.z and b.b.
template <typename T, bool MF>
static __global__ void __launch_bounds__(CAM_THREADS)
k_cam_combine_schur(int C, const int32_t* __restrict__ cam_piece_ptr, const double* __restrict__ part,
                    const double* __restrict__ U, const double* __restrict__ gc, const T* __restrict__ camtab,
                    const double* __restrict__ lam_ptr, double dmin, double dmax, double* __restrict__ Minv,
                    double* __restrict__ x, double* __restrict__ r, double* __restrict__ z,
                    double* __restrict__ p, T* __restrict__ pT, double* __restrict__ dot_rz1,
                    double* __restrict__ dot_bb, const uint8_t* __restrict__ fixed, DevState* st,
                    double* __restrict__ Sii_out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double rz = 0.0, bb = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->pcg_done = 0;
    st->pcg_iters = 0;
    st->pcg_rel = 1.0;
    st->fallbacks = 0;
  }
  if (c < C) {
    int fb;
    cam_schur_one<T, MF>(cam_piece_ptr[c], cam_piece_ptr[c + 1], part, U + 45LL * c, gc + 9LL * c,
                         camtab + (long long)CT * c, *lam_ptr, dmin, dmax, fixed ? fixed + 9LL * c : nullptr,
                         Minv + 45LL * c, x + 9LL * c, r + 9LL * c, z + 9LL * c, p + 9LL * c,
                         pT + (long long)pass_vec_stride(MF) * c, rz, bb, fb,
                         Sii_out ? Sii_out + 45LL * c : nullptr);
    if (fb) atomicAdd(&st->fallbacks, 1);
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

// Pass A, step 1 (camera-major, one CTA per piece of camera c):
//   z_s = Jp_s^T (Jc_s x_c)   for every observation s of the piece,
// written as one 4-vector per observation in camera-major order (coalesced).  The
// camera's table and x_c sit in registers; the only per-observation loads are
// the point index, the point (recompute mode: one 16-byte vector) or the
// planes (stored mode), and sqrt(w).
// z = Jp^T (Jc x) of one observation in the recompute mode: the camera
// table's first 15 entries in ct, the camera vector in the passes' form in xv.
template <typename T, typename CT15, typename XV9>
__device__ __forceinline__ void a1_obs(const CT15& ct, const XV9& xv, T X0, T X1, T X2, T sw, T& z0, T& z1,
                                       T& z2) {
  Fac<T> o;
  fac_obs(ct, X0, X1, X2, sw, o);
  T e0, e1;
  jc_times_fac(o, xv, e0, e1);
  const T a0 = o.A[0] * e0 + o.A[3] * e1;
  const T a1 = o.A[1] * e0 + o.A[4] * e1;
  const T a2 = o.A[2] * e0 + o.A[5] * e1;
  z0 = ct[0] * a0 + ct[3] * a1 + ct[6] * a2;
  z1 = ct[1] * a0 + ct[4] * a1 + ct[7] * a2;
  z2 = ct[2] * a0 + ct[5] * a1 + ct[8] * a2;
}

template <typename T, bool MF, int NT>
__device__ __forceinline__ void pass_a1_range(int beg, int end, const int32_t* __restrict__ cm_pt,
                                              const T* __restrict__ Jcm, const T* __restrict__ cm_sw,
                                              const T* __restrict__ ptab, const T (&ctl)[15], const T (&xl)[9],
                                              int O, T* __restrict__ zbuf) {
  if (MF) {
    // one observation of lookahead: the next point is loaded while this one
    // is computed
    int s = beg + threadIdx.x;
    T X0 = 0, X1 = 0, X2 = 0, sw = 1, pad;
    if (s < end) {
      load4(ptab + 8LL * cm_pt[s], X0, X1, X2, pad);
      if (cm_sw) sw = cm_sw[s];
    }
    while (s < end) {
      const int sn = s + NT;
      T Y0 = 0, Y1 = 0, Y2 = 0, swn = 1;
      if (sn < end) {
        load4(ptab + 8LL * cm_pt[sn], Y0, Y1, Y2, pad);
        if (cm_sw) swn = cm_sw[sn];
      }
      T z0, z1, z2;
      a1_obs(ctl, xl, X0, X1, X2, sw, z0, z1, z2);
      store4(zbuf + 4LL * s, z0, z1, z2, T(0));
      s = sn;
      X0 = Y0;
      X1 = Y1;
      X2 = Y2;
      sw = swn;
    }
  } else {
    for (int s = beg + threadIdx.x; s < end; s += NT) {
      T pl[NPLANE];
      load_planes(Jcm, O, s, pl);
      T j0[9], j1[9];
      jc_rows(pl, j0, j1);
      T e0 = 0, e1 = 0;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        e0 += j0[i] * xl[i];
        e1 += j1[i] * xl[i];
      }
      // z = Jp^T e with the stored Jp = A R
      const T* Jp = pl + NPLANE_JC;
      const T z0 = Jp[0] * e0 + Jp[3] * e1;
      const T z1 = Jp[1] * e0 + Jp[4] * e1;
      const T z2 = Jp[2] * e0 + Jp[5] * e1;
      store4(zbuf + 4LL * s, z0, z1, z2, T(0));
    }
  }
}

template <typename T, bool MF>
static __global__ void __launch_bounds__(PIECE_THREADS)
k_pass_a1(const int32_t* __restrict__ piece_cam, const int32_t* __restrict__ piece_beg,
          const int32_t* __restrict__ piece_end, const int32_t* __restrict__ cm_pt,
          const T* __restrict__ Jcm, const T* __restrict__ cm_sw, const T* __restrict__ ptab,
          const T* __restrict__ camtab, const T* __restrict__ xc, const DevState* __restrict__ st,
          int check_done, int O, T* __restrict__ zbuf) {
  if (check_done && st->pcg_done) return;
  __shared__ T sct[16];
  __shared__ T sx[PV];
  const int b = blockIdx.x;
  const int c = piece_cam[b];
  constexpr int XS = pass_vec_stride(MF);
  if (threadIdx.x < 16) sct[threadIdx.x] = camtab[(long long)CT * c + threadIdx.x];
  if (threadIdx.x >= 32 && threadIdx.x < 32 + XS) sx[threadIdx.x - 32] = xc[(long long)XS * c + threadIdx.x - 32];
  __syncthreads();
  T ctl[15], xl[9];
#pragma unroll
  for (int i = 0; i < 15; ++i) ctl[i] = sct[i];
#pragma unroll
  for (int i = 0; i < 9; ++i) xl[i] = sx[i];
  pass_a1_range<T, MF, PIECE_THREADS>(piece_beg[b], piece_end[b], cm_pt, Jcm, cm_sw, ptab, ctl, xl, O, zbuf);
}

template <typename T, int MODE>
__device__ __forceinline__ double pass_a_point(int j, int P, T z0, T z1, T z2, const T* __restrict__ Vinv,
                                               T* __restrict__ ptab, T* __restrict__ dp, const T* __restrict__ y0,
                                               const double* __restrict__ gp, T* __restrict__ pts_buf, int cur) {
  const T* vi = Vinv + 6LL * j;
  const T t0 = vi[0] * z0 + vi[1] * z1 + vi[2] * z2;
  const T t1 = vi[1] * z0 + vi[3] * z1 + vi[4] * z2;
  const T t2 = vi[2] * z0 + vi[4] * z1 + vi[5] * z2;
  if (MODE == 0) {
    store4(ptab + 8LL * j + 4, t0, t1, t2, T(0));
    return 0.0;
  }
  const T d0 = -(y0[3LL * j] + t0), d1 = -(y0[3LL * j + 1] + t1), d2 = -(y0[3LL * j + 2] + t2);
  dp[3LL * j] = d0;
  dp[3LL * j + 1] = d1;
  dp[3LL * j + 2] = d2;
  const T* src = pts_buf + (long long)cur * 3 * P + 3LL * j;
  T* dst = pts_buf + (long long)(1 - cur) * 3 * P + 3LL * j;
  dst[0] = src[0] + d0;
  dst[1] = src[1] + d1;
  dst[2] = src[2] + d2;
  return gp[3LL * j] * (double)d0 + gp[3LL * j + 1] * (double)d1 + gp[3LL * j + 2] * (double)d2;
}

// Pass A, step 2 (point-major, one CTA per chunk of points):
//   t_j = V*_j^{-1} sum_{k in pt j} z_k
// (one observation per thread gathers its z_k through the point-to-camera
// order map into shared memory; one thread per point adds them in slot
// order).  MODE 0 writes t_j into the point table for pass B; MODE 1
// (back-substitution, z from dc) forms dp_j = -(y0_j + t_j), writes the
// trial point theta_p + dp_j and reduces gp_j . dp_j per chunk.
template <typename T, int MODE>
static __global__ void __launch_bounds__(CHUNK_THREADS)
k_pass_a2(const int32_t* __restrict__ pchunk, int P, const int32_t* __restrict__ rowptr_pt,
          const int32_t* __restrict__ pm2cm, const T* __restrict__ zbuf, const T* __restrict__ Vinv,
          const DevState* __restrict__ st, int check_done, T* __restrict__ ptab, T* __restrict__ dp,
          const T* __restrict__ y0, const double* __restrict__ gp, T* __restrict__ pts_buf,
          double* __restrict__ dot_gp) {
  if (MODE == 0 && check_done && st->pcg_done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sz = reinterpret_cast<T*>(smem_raw);  // [CHUNK_SLOTS][4]
  const int cur = st->cur;
  const int j0 = pchunk[blockIdx.x], j1 = pchunk[blockIdx.x + 1];
  const int s0 = rowptr_pt[j0], s1 = rowptr_pt[j1];
  double gd = 0.0;
  if (s1 - s0 <= CHUNK_SLOTS) {
    // all gathers of this thread in flight at once
    // all gathers of this thread in flight at once
    constexpr int U = CHUNK_SLOTS / CHUNK_THREADS;
    int src[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int q = s0 + threadIdx.x + u * CHUNK_THREADS;
      src[u] = q < s1 ? pm2cm[q] : -1;
    }
    T zz[U][4];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (src[u] >= 0) load4(zbuf + 4LL * src[u], zz[u][0], zz[u][1], zz[u][2], zz[u][3]);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (src[u] >= 0) store4(sz + 4 * (threadIdx.x + u * CHUNK_THREADS), zz[u][0], zz[u][1], zz[u][2], zz[u][3]);
    __syncthreads();
    for (int j = j0 + threadIdx.x; j < j1; j += CHUNK_THREADS) {
      T z0 = 0, z1 = 0, z2 = 0;
      const int q1 = rowptr_pt[j + 1];
      for (int q = rowptr_pt[j]; q < q1; ++q) {
        T a, b, c, pad;
        load4(sz + 4 * (q - s0), a, b, c, pad);
        z0 += a;
        z1 += b;
        z2 += c;
      }
      gd += pass_a_point<T, MODE>(j, P, z0, z1, z2, Vinv, ptab, dp, y0, gp, pts_buf, cur);
    }
  } else {
    T z0 = 0, z1 = 0, z2 = 0;
    for (int q = s0 + threadIdx.x; q < s1; q += CHUNK_THREADS) {
      T a, b, c, d;
      load4(zbuf + 4LL * pm2cm[q], a, b, c, d);
      z0 += a;
      z1 += b;
      z2 += c;
    }
    double dd[3] = {(double)z0, (double)z1, (double)z2};
    block_sum_all<3>(dd);
    if (threadIdx.x == 0)
      gd = pass_a_point<T, MODE>(j0, P, (T)dd[0], (T)dd[1], (T)dd[2], Vinv, ptab, dp, y0, gp, pts_buf, cur);
  }
  if (MODE == 1) {
    double v[1] = {gd};
    block_sum_all<1>(v);
    if (threadIdx.x == 0) dot_gp[blockIdx.x] = v[0];
  }
}

// Fused pass A (recompute mode, point-major, one CTA per chunk of points):
//   t_j = V*_j^{-1} sum_{k in pt j} Jp_k^T (Jc_k x_c(k))
// in one kernel.  The points of a chunk are seen by few cameras (points are
// numbered by their first camera): the chunk's cameras -- their tables and
// vectors x_c -- are staged in shared memory (at most FA_CAMS of them, the
// list built in the symbolic phase, pm_lc the position of each slot's camera
// in it; the staging area is sized by nc_max, the most cameras any chunk of
// the problem sees, which leaves the rest of the SM's carveout to L1 for the
// point gathers), so no per-observation camera data and no per-observation
// intermediate leave the SM.  Each thread issues all loads of its slots and
// of its point before the first barrier.  The per-observation products and
// the per-point sums are those of passes A1 and A2 (same order).  MODE as in
// k_pass_a2.  SW = false (no robust loss, sqrt(w) = 1) compiles the weight's
// loads and products out; the results are the same bits.

template <typename T, int MODE, bool SW = true>
static __global__ void __launch_bounds__(CHUNK_THREADS, sizeof(T) == 4 ? 5 : 1)
k_pass_fa(const int32_t* __restrict__ pchunk, int P, const int32_t* __restrict__ rowptr_pt,
          const int32_t* __restrict__ pm_pt, const int16_t* __restrict__ pm_lc, const T* __restrict__ pm_sw,
          const int32_t* __restrict__ chunk_cams, const int32_t* __restrict__ chunk_cam_ptr,
          const T* __restrict__ camtab, const T* __restrict__ xc, const T* __restrict__ Vinv,
          const DevState* __restrict__ st, int check_done, T* __restrict__ ptab, T* __restrict__ dp,
          const T* __restrict__ y0, const double* __restrict__ gp, T* __restrict__ pts_buf,
          double* __restrict__ dot_gp, const int4* __restrict__ chunk_hdr, int nc_max) {
  if (MODE == 0 && check_done && st->pcg_done) return;
  if (!SW) pm_sw = nullptr;  // no robust loss: sqrt(w) = 1 folds away
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sz = reinterpret_cast<T*>(smem_raw);  // [CHUNK_SLOTS][4]
  T* sX = sz + 4 * CHUNK_SLOTS;            // [CHUNK_PTS][4]: the chunk's points
  T* sct = sX + 4 * CHUNK_PTS;             // [nc_max][FA_CT]: camera tables
  T* sxv = sct + nc_max * FA_CT;           // [nc_max][FA_XV]: camera vectors
  constexpr int U = CHUNK_SLOTS / CHUNK_THREADS;
  const int k = blockIdx.x;
  // the chunk's header: first/last point and slot, camera list, and the
  // first camera when the list is a contiguous range (else -1), so every
  // other load of the kernel depends on this one only
  const int4 h0 = chunk_hdr[2 * k], h1 = chunk_hdr[2 * k + 1];
  const int j0 = h0.x, j1 = h0.y, s0 = h0.z, s1 = h0.w, c0 = h1.x, nc = h1.y, cmin = h1.z;
  const bool small = s1 - s0 <= CHUNK_SLOTS;
  // this thread's slots: their point, camera position and sqrt(w)
  int jj[U], ll[U];
  T sw[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int q = s0 + threadIdx.x + u * CHUNK_THREADS;
    const bool v = small && q < s1;
    jj[u] = v ? pm_pt[q] : -1;
    ll[u] = v ? pm_lc[q] : 0;
    sw[u] = (v && pm_sw) ? pm_sw[q] : T(1);
  }
  // this thread's first point: its slot range and V*^{-1}
  const int jp = j0 + threadIdx.x;
  int p0 = 0, p1 = 0;
  T vi[6] = {};
  if (small && jp < j1) {
    p0 = rowptr_pt[jp];
    p1 = rowptr_pt[jp + 1];
#pragma unroll
    for (int i = 0; i < 6; ++i) vi[i] = Vinv[6LL * jp + i];
  }
  // the chunk's points are contiguous: their X, one coalesced row each, not
  // a gather behind the slot's point index
  if (small) {
    for (int p = threadIdx.x; p < j1 - j0; p += CHUNK_THREADS) {
      T a, b, c, pad;
      load4(ptab + 8LL * (j0 + p), a, b, c, pad);
      store4(sX + 4 * p, a, b, c, T(0));
    }
  }
  for (int i = threadIdx.x; i < nc * 16; i += CHUNK_THREADS) {
    const int l = i >> 4, e = i & 15;
    const int cam = cmin >= 0 ? cmin + l : chunk_cams[c0 + l];
    if (e < 15) sct[l * FA_CT + e] = camtab[(long long)CT * cam + e];
  }
  for (int i = threadIdx.x; i < nc * 9; i += CHUNK_THREADS) {
    const int l = i / 9, e = i % 9;
    const int cam = cmin >= 0 ? cmin + l : chunk_cams[c0 + l];
    sxv[l * FA_XV + e] = xc[(long long)PV * cam + e];
  }
  __syncthreads();
  const int cur = st->cur;
  double gd = 0.0;
  if (small) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (jj[u] < 0) continue;
      T X0, X1, X2, pad;
      load4(sX + 4 * (jj[u] - j0), X0, X1, X2, pad);
      T z0, z1, z2;
      a1_obs(sct + ll[u] * FA_CT, sxv + ll[u] * FA_XV, X0, X1, X2, sw[u], z0, z1, z2);
      store4(sz + 4 * (threadIdx.x + u * CHUNK_THREADS), z0, z1, z2, T(0));
    }
    __syncthreads();
    for (int j = jp; j < j1; j += CHUNK_THREADS) {
      if (j != jp) {
        p0 = rowptr_pt[j];
        p1 = rowptr_pt[j + 1];
      }
      T z0 = 0, z1 = 0, z2 = 0;
      for (int q = p0; q < p1; ++q) {
        T a, b, c, pad;
        load4(sz + 4 * (q - s0), a, b, c, pad);
        z0 += a;
        z1 += b;
        z2 += c;
      }
      if (j == jp && MODE == 0) {
        // V*^{-1} already in registers: t_j as in pass_a_point
        const T t0 = vi[0] * z0 + vi[1] * z1 + vi[2] * z2;
        const T t1 = vi[1] * z0 + vi[3] * z1 + vi[4] * z2;
        const T t2 = vi[2] * z0 + vi[4] * z1 + vi[5] * z2;
        store4(ptab + 8LL * j + 4, t0, t1, t2, T(0));
      } else {
        gd += pass_a_point<T, MODE>(j, P, z0, z1, z2, Vinv, ptab, dp, y0, gp, pts_buf, cur);
      }
    }
  } else {
    T z0 = 0, z1 = 0, z2 = 0;
    for (int q = s0 + threadIdx.x; q < s1; q += CHUNK_THREADS) {
      const int l = pm_lc[q];
      T X0, X1, X2, pad;
      load4(ptab + 8LL * pm_pt[q], X0, X1, X2, pad);
      T a, b, c;
      a1_obs(sct + l * FA_CT, sxv + l * FA_XV, X0, X1, X2, pm_sw ? pm_sw[q] : T(1), a, b, c);
      z0 += a;
      z1 += b;
      z2 += c;
    }
    double dd[3] = {(double)z0, (double)z1, (double)z2};
    block_sum_all<3>(dd);
    if (threadIdx.x == 0)
      gd = pass_a_point<T, MODE>(j0, P, (T)dd[0], (T)dd[1], (T)dd[2], Vinv, ptab, dp, y0, gp, pts_buf, cur);
  }
  if (MODE == 1) {
    double v[1] = {gd};
    block_sum_all<1>(v);
    if (threadIdx.x == 0) dot_gp[blockIdx.x] = v[0];
  }
}

// ---------------------------------------------------------------------------
// Stored mode: pass A fused point-major (A1 + A2 in one kernel)
// ---------------------------------------------------------------------------

// The stored planes in point-major slot order: Jpm[q] = Jcm[pm2cm[q]] (both
// pair-interleaved), gathered once per linearisation (gated like it).
template <typename T>
static __global__ void k_planes_pm(long long O, const DevState* __restrict__ st, int gate,
                                   const int32_t* __restrict__ pm2cm, const T* __restrict__ Jcm,
                                   T* __restrict__ Jpm) {
  if (gate && !st->need_lin) return;
  using V2 = typename Vec2<T>::type;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= O) return;
  const long long s = pm2cm[q];
#pragma unroll
  for (int p = 0; p < NPLANE / 2; ++p)
    reinterpret_cast<V2*>(Jpm)[p * O + q] = reinterpret_cast<const V2*>(Jcm)[p * O + s];
}

// Fused pass A of the stored mode (point-major, one CTA per chunk of
// points):  t_j = V*_j^{-1} sum_{k in pt j} Jp_k^T (Jc_k x_c(k)),  the
// products of k_pass_a1 on the point-major copy of the planes, the chunk's
// camera vectors staged in shared memory (the chunk lists of k_pass_fa),
// and the per-point sums of k_pass_a2 in slot order -- without the
// per-observation z written to and gathered back from global memory.  A
// chunk of one point with more than CHUNK_SLOTS observations is reduced by
// the block.
template <typename T>
static __global__ void __launch_bounds__(CHUNK_THREADS)
k_pass_fs(const int32_t* __restrict__ rowptr_pt, const int16_t* __restrict__ pm_lc,
          const int32_t* __restrict__ chunk_cams, const T* __restrict__ Jpm, long long O, const T* __restrict__ xc,
          const T* __restrict__ Vinv, const DevState* __restrict__ st, int check_done, T* __restrict__ ptab,
          const int4* __restrict__ chunk_hdr, int nc_max) {
  if (check_done && st->pcg_done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sz = reinterpret_cast<T*>(smem_raw);  // [CHUNK_SLOTS][4]
  T* sxv = sz + 4 * CHUNK_SLOTS;           // [nc_max][9]: the chunk's camera vectors
  const int k = blockIdx.x;
  const int4 h0 = chunk_hdr[2 * k], h1 = chunk_hdr[2 * k + 1];
  const int j0 = h0.x, j1 = h0.y, s0 = h0.z, s1 = h0.w, c0 = h1.x, nc = h1.y, cmin = h1.z;
  const bool small = s1 - s0 <= CHUNK_SLOTS;
  for (int i = threadIdx.x; i < nc * 9; i += CHUNK_THREADS) {
    const int l = i / 9, e = i % 9;
    const int cam = cmin >= 0 ? cmin + l : chunk_cams[c0 + l];
    sxv[i] = xc[9LL * cam + e];
  }
  __syncthreads();
  T za = 0, zb = 0, zc = 0;  // large chunk: this thread's share
  for (int q = s0 + threadIdx.x; q < s1; q += CHUNK_THREADS) {
    T pl[NPLANE];
    load_planes(Jpm, O, q, pl);
    const T* xv = sxv + 9 * pm_lc[q];
    T j0r[9], j1r[9];
    jc_rows(pl, j0r, j1r);
    T e0 = 0, e1 = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      e0 += j0r[i] * xv[i];
      e1 += j1r[i] * xv[i];
    }
    const T* Jp = pl + NPLANE_JC;
    const T z0 = Jp[0] * e0 + Jp[3] * e1;
    const T z1 = Jp[1] * e0 + Jp[4] * e1;
    const T z2 = Jp[2] * e0 + Jp[5] * e1;
    if (small) {
      store4(sz + 4 * (q - s0), z0, z1, z2, T(0));
    } else {
      za += z0;
      zb += z1;
      zc += z2;
    }
  }
  if (small) {
    __syncthreads();
    for (int j = j0 + threadIdx.x; j < j1; j += CHUNK_THREADS) {
      T z0 = 0, z1 = 0, z2 = 0;
      const int q1 = rowptr_pt[j + 1];
      for (int q = rowptr_pt[j]; q < q1; ++q) {
        T a, b, c, pad;
        load4(sz + 4 * (q - s0), a, b, c, pad);
        z0 += a;
        z1 += b;
        z2 += c;
      }
      const T* vi = Vinv + 6LL * j;
      const T t0 = vi[0] * z0 + vi[1] * z1 + vi[2] * z2;
      const T t1 = vi[1] * z0 + vi[3] * z1 + vi[4] * z2;
      const T t2 = vi[2] * z0 + vi[4] * z1 + vi[5] * z2;
      store4(ptab + 8LL * j + 4, t0, t1, t2, T(0));
    }
  } else {
    double dd[3] = {(double)za, (double)zb, (double)zc};
    block_sum_all<3>(dd);
    if (threadIdx.x == 0) {
      const T* vi = Vinv + 6LL * j0;
      const T z0 = (T)dd[0], z1 = (T)dd[1], z2 = (T)dd[2];
      store4(ptab + 8LL * j0 + 4, vi[0] * z0 + vi[1] * z1 + vi[2] * z2, vi[1] * z0 + vi[3] * z1 + vi[4] * z2,
             vi[2] * z0 + vi[4] * z1 + vi[5] * z2, T(0));
    }
  }
}

// dynamic shared memory of k_pass_fs: z per slot and nc camera vectors
template <typename T>
constexpr int fs_smem(int nc) {
  return (CHUNK_SLOTS * 4 + nc * 9) * (int)sizeof(T);
}

// Pass B over camera-major slots [beg, end), NT threads striding: per-thread
// partial sum_k Jc_k^T (Jp_k t_p(k)) (9 values; in the recompute mode the
// first three are still to be multiplied by J_l^T).
template <typename T, bool MF, int NT, int UB = 1, bool PF = false>
__device__ __forceinline__ void pass_b_range(int beg, int end, const int32_t* __restrict__ cm_pt,
                                             const T* __restrict__ Jcm, const T* __restrict__ cm_sw,
                                             const T* __restrict__ ptab, const T (&ctl)[15], int O, T (&acc)[9]) {
  if (MF && UB > 1) {
    // UB slots per thread and round: all index loads, then all point
    // gathers, then the products (UB gathers in flight per thread); with
    // PF the next round's indices are loaded before this round's gathers
    int jn[UB];
    T swn[UB];
    if (PF) {
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        const int s = beg + threadIdx.x + u * NT;
        jn[u] = s < end ? cm_pt[s] : -1;
        swn[u] = (s < end && cm_sw) ? cm_sw[s] : T(1);
      }
    }
    for (int s0 = beg + threadIdx.x; s0 < end; s0 += UB * NT) {
      int j[UB];
      T sw[UB], X[UB][3], t[UB][3];
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        if (PF) {
          j[u] = jn[u];
          sw[u] = swn[u];
          const int s = s0 + (UB + u) * NT;
          jn[u] = s < end ? cm_pt[s] : -1;
          swn[u] = (s < end && cm_sw) ? cm_sw[s] : T(1);
        } else {
          const int s = s0 + u * NT;
          j[u] = s < end ? cm_pt[s] : -1;
          sw[u] = (s < end && cm_sw) ? cm_sw[s] : T(1);
        }
      }
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        T pad;
        if (j[u] >= 0) {
          load4(ptab + 8LL * j[u], X[u][0], X[u][1], X[u][2], pad);
          load4(ptab + 8LL * j[u] + 4, t[u][0], t[u][1], t[u][2], pad);
        }
      }
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        if (j[u] < 0) continue;
        const T g0 = ctl[0] * t[u][0] + ctl[1] * t[u][1] + ctl[2] * t[u][2];
        const T g1 = ctl[3] * t[u][0] + ctl[4] * t[u][1] + ctl[5] * t[u][2];
        const T g2 = ctl[6] * t[u][0] + ctl[7] * t[u][1] + ctl[8] * t[u][2];
        Fac<T> o;
        fac_obs(ctl, X[u][0], X[u][1], X[u][2], sw[u], o);
        const T h0 = o.A[0] * g0 + o.A[1] * g1 + o.A[2] * g2;
        const T h1 = o.A[3] * g0 + o.A[4] * g1 + o.A[5] * g2;
        jct_fac_acc(o, h0, h1, acc);
      }
    }
  } else if (MF) {
    int s = beg + threadIdx.x;
    T X0 = 0, X1 = 0, X2 = 0, t0 = 0, t1 = 0, t2 = 0, sw = 1, pad;
    if (s < end) {
      const int j = cm_pt[s];
      load4(ptab + 8LL * j, X0, X1, X2, pad);
      load4(ptab + 8LL * j + 4, t0, t1, t2, pad);
      if (cm_sw) sw = cm_sw[s];
    }
    while (s < end) {
      const int sn = s + NT;
      T Y0 = 0, Y1 = 0, Y2 = 0, u0 = 0, u1 = 0, u2 = 0, swn = 1;
      if (sn < end) {
        const int jn = cm_pt[sn];
        load4(ptab + 8LL * jn, Y0, Y1, Y2, pad);
        load4(ptab + 8LL * jn + 4, u0, u1, u2, pad);
        if (cm_sw) swn = cm_sw[sn];
      }
      const T g0 = ctl[0] * t0 + ctl[1] * t1 + ctl[2] * t2;
      const T g1 = ctl[3] * t0 + ctl[4] * t1 + ctl[5] * t2;
      const T g2 = ctl[6] * t0 + ctl[7] * t1 + ctl[8] * t2;
      Fac<T> o;
      fac_obs(ctl, X0, X1, X2, sw, o);
      const T h0 = o.A[0] * g0 + o.A[1] * g1 + o.A[2] * g2;
      const T h1 = o.A[3] * g0 + o.A[4] * g1 + o.A[5] * g2;
      jct_fac_acc(o, h0, h1, acc);
      s = sn;
      X0 = Y0;
      X1 = Y1;
      X2 = Y2;
      t0 = u0;
      t1 = u1;
      t2 = u2;
      sw = swn;
    }
  } else {
    for (int s = beg + threadIdx.x; s < end; s += NT) {
      const int j = cm_pt[s];
      T t0, t1, t2, tpad;
      load4(ptab + 8LL * j + 4, t0, t1, t2, tpad);
      T pl[NPLANE];
      load_planes(Jcm, O, s, pl);
      // h = Jp t with the stored Jp = A R
      const T* Jp = pl + NPLANE_JC;
      const T h0 = Jp[0] * t0 + Jp[1] * t1 + Jp[2] * t2;
      const T h1 = Jp[3] * t0 + Jp[4] * t1 + Jp[5] * t2;
      T j0[9], j1[9];
      jc_rows(pl, j0, j1);
      // two fused multiply-adds per component
#pragma unroll
      for (int i = 0; i < 9; ++i) acc[i] = fma(j1[i], h1, fma(j0[i], h0, acc[i]));
    }
  }
}

// Pass B (camera-major): per piece, sum_k Jc_k^T (Jp_k t_p(k)); UB, PF as in
// pass_b_range.  NT threads per piece: the FP32 recompute mode runs 128
// (16 slots per thread, the per-piece reduction amortised over twice the
// work of a 256-thread CTA; 8 CTAs per SM at the same 64-register cap).
// SW as in k_pass_fa.
template <typename T, bool MF, int UB = 1, bool PF = false, int NT = PIECE_THREADS, bool SW = true>
static __global__ void __launch_bounds__(NT, UB > 1 ? 1024 / NT : 1)
k_pass_b(const int32_t* __restrict__ piece_cam, const int32_t* __restrict__ piece_beg,
         const int32_t* __restrict__ piece_end, const int32_t* __restrict__ cm_pt,
         const T* __restrict__ Jcm, const T* __restrict__ cm_sw, const T* __restrict__ ptab,
         const T* __restrict__ camtab, const DevState* __restrict__ st, int check_done, int O,
         double* __restrict__ part) {
  if (check_done && st->pcg_done) return;
  if (!SW) cm_sw = nullptr;  // no robust loss: sqrt(w) = 1 folds away
  __shared__ T sct[16];
  const int b = blockIdx.x;
  const int c = piece_cam[b];
  if (threadIdx.x < 16) sct[threadIdx.x] = camtab[(long long)CT * c + threadIdx.x];
  __syncthreads();
  T ctl[15];
#pragma unroll
  for (int i = 0; i < 15; ++i) ctl[i] = sct[i];
  T acc[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) acc[i] = T(0);
  pass_b_range<T, MF, NT, UB, PF>(piece_beg[b], piece_end[b], cm_pt, Jcm, cm_sw, ptab, ctl, O, acc);
  block_sum_store<9, false>(acc, part + (long long)PART * b);
}

// The per-iteration vector kernels run 9 threads per camera (one per
// component), CAM_THREADS cameras per block, so the FP64 9x9 products are
// spread over the whole GPU instead of one serial thread per camera.
constexpr int VT = CAM_THREADS * 9;

__device__ __forceinline__ int sym9_rt(int i, int j) { return i <= j ? sym9(i, j) : sym9(j, i); }

// q = U* p - sum of pass-B partials (J_l^T applied to their first three in
// the recompute mode); per-block partial p.q.  Camera c's partials are rows
// cam_piece_ptr[c] .. cam_piece_ptr[c + 1] of part (row stride PS): per
// piece, or one row per camera already summed (a point-partitioned problem).
template <typename T, bool MF, int PS = PART>
static __global__ void __launch_bounds__(VT)
k_pcg_q(int C, const int32_t* __restrict__ cam_piece_ptr, const double* __restrict__ part,
        const double* __restrict__ U, const T* __restrict__ camtab, const double* __restrict__ lam_ptr, double dmin,
        double dmax, const double* __restrict__ p, double* __restrict__ q, double* __restrict__ dot_pq,
        const uint8_t* __restrict__ fixed, const DevState* __restrict__ st, int check_done) {
  if (check_done && st->pcg_done) return;
  __shared__ double sp[CAM_THREADS][9], ss[CAM_THREADS][9];
  const int lc = threadIdx.x / 9, i = threadIdx.x % 9;
  const int c = blockIdx.x * CAM_THREADS + lc;
  const bool ok = c < C;
  double pv = 0.0, sum = 0.0;
  if (ok) {
    pv = p[9LL * c + i];
    const int p1 = cam_piece_ptr[c + 1];
    for (int k = cam_piece_ptr[c]; k < p1; ++k) sum += part[(long long)PS * k + i];
  }
  sp[lc][i] = pv;
  ss[lc][i] = sum;
  __syncthreads();
  double pq = 0.0;
  if (ok) {
    if (MF && i < 3) {
      const T* Jl = camtab + (long long)CT * c + CT_JL;
      sum = (double)Jl[i] * ss[lc][0] + (double)Jl[3 + i] * ss[lc][1] + (double)Jl[6 + i] * ss[lc][2];
    }
    const double* Uc = U + 45LL * c;
    double y = damp(Uc[sym9(i, i)], *lam_ptr, dmin, dmax) * sp[lc][i];
#pragma unroll
    for (int j = 0; j < 9; ++j) y += Uc[sym9_rt(i, j)] * sp[lc][j];
    y -= sum;
    if (fixed && fixed[9LL * c + i]) y = 0.0;
    q[9LL * c + i] = y;
    pq = pv * y;
  }
  double v[1] = {pq};
  block_sum_all<1>(v);
  if (threadIdx.x == 0 && dot_pq) dot_pq[blockIdx.x] = v[0];
}

// alpha = (r.z)_old / p.q; x += alpha p; r -= alpha q; z = M r;
// partial r.z into dot_rz[k & 1], partial r.r.
static __global__ void __launch_bounds__(VT)
k_pcg_update(int C, int nb, int k, const double* __restrict__ dot_pq, double* __restrict__ dot_rz,
             double* __restrict__ dot_rr, const double* __restrict__ p, const double* __restrict__ q,
             double* __restrict__ x, double* __restrict__ r, double* __restrict__ z,
             const double* __restrict__ Minv, DevState* st) {
  if (st->pcg_done) return;
  const double* const srcs[2] = {dot_pq, dot_rz + ((k + 1) & 1) * nb};
  double sums[2];
  block_sum_arrays<2>(srcs, nb, sums);
  const double pq = sums[0], rz_old = sums[1];
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
  __shared__ double sr[CAM_THREADS][9];
  const int lc = threadIdx.x / 9, i = threadIdx.x % 9;
  const int c = blockIdx.x * CAM_THREADS + lc;
  const bool ok = c < C;
  double rv = 0.0;
  if (ok) {
    const long long o = 9LL * c + i;
    x[o] += alpha * p[o];
    rv = r[o] - alpha * q[o];
    r[o] = rv;
  }
  sr[lc][i] = rv;
  __syncthreads();
  double zz = 0.0;
  if (ok) {
    const double* M = Minv + 45LL * c;
#pragma unroll
    for (int j = 0; j < 9; ++j) zz += M[sym9_rt(i, j)] * sr[lc][j];
    z[9LL * c + i] = zz;
  }
  double v[2] = {rv * zz, rv * rv};
  block_sum_all<2>(v);
  if (threadIdx.x == 0) {
    dot_rz[(k & 1) * nb + blockIdx.x] = v[0];
    dot_rr[blockIdx.x] = v[1];
  }
}

// Convergence test |r| <= tol |b|; beta = (r.z)_new / (r.z)_old; p = z + beta p,
// and p in the passes' form.
template <typename T, bool MF>
static __global__ void __launch_bounds__(VT)
k_pcg_direction(int C, int nb, int k, double tol, const double* __restrict__ dot_rz,
                const double* __restrict__ dot_rr, const double* __restrict__ dot_bb,
                const double* __restrict__ z, double* __restrict__ p, const T* __restrict__ camtab,
                T* __restrict__ pT, DevState* st) {
  if (st->pcg_done) return;
  const double* const srcs[4] = {dot_rz + (k & 1) * nb, dot_rz + ((k + 1) & 1) * nb, dot_rr, dot_bb};
  double sums[4];
  block_sum_arrays<4>(srcs, nb, sums);
  const double rz_new = sums[0], rz_old = sums[1], rr = sums[2], bb = sums[3];
  const bool conv = sqrt(rr) <= tol * sqrt(bb);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->pcg_iters = k + 1;
    st->pcg_rel = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    if (conv) st->pcg_done = 1;
  }
  if (conv) return;
  const double beta = rz_new / rz_old;
  __shared__ double sp[CAM_THREADS][9];
  const int lc = threadIdx.x / 9, i = threadIdx.x % 9;
  const int c = blockIdx.x * CAM_THREADS + lc;
  const bool ok = c < C;
  double pv = 0.0;
  if (ok) {
    const long long o = 9LL * c + i;
    pv = z[o] + beta * p[o];
    p[o] = pv;
  }
  sp[lc][i] = pv;
  __syncthreads();
  if (!ok) return;
  constexpr int XS = pass_vec_stride(MF);
  T* out = pT + (long long)XS * c;
  if (MF && i < 3) {
    const T* Jl = camtab + (long long)CT * c + CT_JL;
    out[i] = (T)((double)Jl[3 * i] * sp[lc][0] + (double)Jl[3 * i + 1] * sp[lc][1] + (double)Jl[3 * i + 2] * sp[lc][2]);
    out[9 + i] = T(0);
  } else {
    out[i] = (T)pv;
  }
}

// ---------------------------------------------------------------------------
// a5 / a6: trial parameters, trial cost, model reduction, LM control
// ---------------------------------------------------------------------------

// One trial camera dst = src + dc (dc rounded to T), dc in the pass form;
// returns gc . dc.
template <typename T, bool MF>
__device__ __forceinline__ double cam_trial_one(const double* __restrict__ xc, const double* __restrict__ gcc,
                                                const T* __restrict__ src, T* __restrict__ dst,
                                                const T* __restrict__ ct, T* __restrict__ xTc) {
  double gd = 0.0;
  double dr[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const T d = (T)xc[i];
    dr[i] = (double)d;
    dst[i] = src[i] + d;
    gd += gcc[i] * (double)d;
  }
  write_pass_vec<T, MF>(ct, dr, xTc);
  return gd;
}

// Trial cameras theta_c + dc (dc rounded to T), dc in the pass form, partial
// gc . dc.
template <typename T, bool MF>
static __global__ void __launch_bounds__(CAM_THREADS)
k_cam_trial(int C, const double* __restrict__ x, const double* __restrict__ gc, T* __restrict__ cams_buf,
            const T* __restrict__ camtab, const DevState* __restrict__ st, T* __restrict__ xT,
            double* __restrict__ dot_gc) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double gd = 0.0;
  if (c < C) {
    const int cur = st->cur;
    gd = cam_trial_one<T, MF>(x + 9LL * c, gc + 9LL * c, cams_buf + (long long)cur * 9 * C + 9LL * c,
                              cams_buf + (long long)(1 - cur) * 9 * C + 9LL * c, camtab + (long long)CT * c,
                              xT + (long long)pass_vec_stride(MF) * c);
  }
  double v[1] = {gd};
  block_sum_all<1>(v);
  if (threadIdx.x == 0) dot_gc[blockIdx.x] = v[0];
}

// Cost terms over camera-major slots [beg, end), NT threads striding:
// 1/2 rho at the camera table sct and points pts, and with MODEL the
// quadratic model term |Jc dc + Jp dp|^2 at the linearisation (camera table
// sold, points pts_old, dc in the pass form sdc).
// The cost 1/2 sum rho is evaluated to about FP64 accuracy in both
// precisions (the accept / reject test and the gain ratio compare costs
// that differ by less than FP32 evaluation would resolve: a robust loss
// converges linearly, and its last gains are ~1e-8 relative per trial).
// FP64: in double with the camera table sct64.  FP32: the squared residual
// in float-float arithmetic on the FP32 pipes from the split table ffc (the
// FP32 parameters and pixels are exact in it), then rho and the sum in
// double.  The model term stays in T, summed in float-float for FP32.
template <typename T, bool MODEL, bool MF, int NT>
__device__ __forceinline__ void cost_cam_range(int beg, int end, const int32_t* __restrict__ cm_pt,
                                               const T* __restrict__ cm_px, const T* __restrict__ pts,
                                               const T* __restrict__ pts_old, const FFCam* __restrict__ ffc,
                                               const double* __restrict__ sct64, const T* __restrict__ sold,
                                               const T* __restrict__ sdc, T delta, int O,
                                               const T* __restrict__ Jcm, const T* __restrict__ cm_sw,
                                               const T* __restrict__ dp, double& cost, double& quad) {
  // model term, FP32: per-thread sums in float-float (about 48 bits, on the
  // FP32 pipes; the products exact by fma); FP64: in double
  float qh = 0.f, ql = 0.f;
  for (int s = beg + threadIdx.x; s < end; s += NT) {
    const int j = cm_pt[s];
    {
      double sq = 0.0;
      bool done = false;
      if constexpr (sizeof(T) == 4) {
        sq = sq_residual_ff(*ffc, pts[3LL * j], pts[3LL * j + 1], pts[3LL * j + 2], cm_px[s], cm_px[(long long)O + s]);
        // outside float range (a trial point near the camera plane): in double
        done = isfinite(sq);
      }
      if (!done) {
        double px, py, sc;
        project_obs(sct64, (double)pts[3LL * j], (double)pts[3LL * j + 1], (double)pts[3LL * j + 2], px, py, sc);
        const double r0 = sc * px - (double)cm_px[s], r1 = sc * py - (double)cm_px[(long long)O + s];
        sq = r0 * r0 + r1 * r1;
      }
      double hr, w;
      huber_weight(sq, (double)delta, hr, w);
      cost += hr;
    }
    if (MODEL) {
      const T d0 = dp[3LL * j], d1 = dp[3LL * j + 1], d2 = dp[3LL * j + 2];
      const T g0 = sold[0] * d0 + sold[1] * d1 + sold[2] * d2;
      const T g1 = sold[3] * d0 + sold[4] * d1 + sold[5] * d2;
      const T g2 = sold[6] * d0 + sold[7] * d1 + sold[8] * d2;
      T e0, e1;
      if (MF) {
        Fac<T> o;
        fac_obs(sold, pts_old[3LL * j], pts_old[3LL * j + 1], pts_old[3LL * j + 2], cm_sw ? cm_sw[s] : T(1), o);
        jc_times_fac(o, sdc, e0, e1);
        e0 += o.A[0] * g0 + o.A[1] * g1 + o.A[2] * g2;
        e1 += o.A[3] * g0 + o.A[4] * g1 + o.A[5] * g2;
      } else {
        T pl[NPLANE];
        load_planes<NPLANE_JC>(Jcm, O, s, pl);
        T j0[9], j1[9];
        jc_rows(pl, j0, j1);
        e0 = pl[0] * g0 + pl[1] * g1 + pl[2] * g2;
        e1 = pl[3] * g0 + pl[4] * g1 + pl[5] * g2;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          e0 += j0[i] * sdc[i];
          e1 += j1[i] * sdc[i];
        }
      }
      if constexpr (sizeof(T) == 4) {
        const float p0 = e0 * e0, p1 = e1 * e1;
        ff_add(qh, ql, p0, fmaf(e0, e0, -p0));
        ff_add(qh, ql, p1, fmaf(e1, e1, -p1));
      } else {
        quad += (double)e0 * (double)e0 + (double)e1 * (double)e1;
      }
    }
  }
  if constexpr (sizeof(T) == 4) quad += (double)qh + (double)ql;
}

// Camera-major pass over the pieces: cost 1/2 sum rho at the parameters in
// buffer (which == 0: current, 1: trial), and with MODEL the quadratic term
// sum_k |Jc_k dc + Jp_k dp|^2 of the model reduction (weights folded in).
template <typename T, bool MODEL, bool MF, int NT = PIECE_THREADS>
static __global__ void __launch_bounds__(NT)
k_cost_cam(const int32_t* __restrict__ piece_cam, const int32_t* __restrict__ piece_beg,
           const int32_t* __restrict__ piece_end, const int32_t* __restrict__ cm_pt,
           const T* __restrict__ cm_px, const T* __restrict__ cams_buf, const T* __restrict__ pts_buf,
           const DevState* __restrict__ st, int which, T delta, int C, int P, int O,
           const T* __restrict__ Jcm, const T* __restrict__ cm_sw, const T* __restrict__ camtab,
           const T* __restrict__ xT, const T* __restrict__ dp, double* __restrict__ part) {
  if (which == 2 && !st->need_cost) return;  // cost at theta only if stale
  __shared__ double sct64[CT];  // camera of the evaluated parameters, in double
  __shared__ FFCam sff;         // and split into float-float pairs (FP32)
  __shared__ T sold[CT];  // camera of the linearisation (model term)
  __shared__ T sdc[PV];
  const int b = blockIdx.x;
  const int c = piece_cam[b];
  const int cur = st->cur;
  const int buf = which == 1 ? 1 - cur : cur;
  if (threadIdx.x == 0) {
    camera_table_f64(cams_buf + (long long)buf * 9 * C + 9LL * c, sct64);
    ffcam_from(sct64, sff);
  }
  if (MODEL && threadIdx.x >= 32 && threadIdx.x < 32 + CT)
    sold[threadIdx.x - 32] = camtab[(long long)CT * c + threadIdx.x - 32];
  if (MODEL && threadIdx.x >= 64 + CT && threadIdx.x < 64 + CT + pass_vec_stride(MF))
    sdc[threadIdx.x - 64 - CT] = xT[(long long)pass_vec_stride(MF) * c + threadIdx.x - 64 - CT];
  __syncthreads();
  const T* pts = pts_buf + (long long)buf * 3 * P;
  const T* pts_old = pts_buf + (long long)cur * 3 * P;
  double cost = 0.0, quad = 0.0;
  static_assert(NT >= 64 + CT + PV, "the staging of the model term needs 64 + CT + PV threads");
  cost_cam_range<T, MODEL, MF, NT>(piece_beg[b], piece_end[b], cm_pt, cm_px, pts, pts_old, &sff, sct64, sold, sdc,
                                   delta, O, Jcm, cm_sw, dp, cost, quad);
  double v[2] = {cost, quad};
  block_sum_store<2>(v, part + (long long)PART * b);
}

// ---------------------------------------------------------------------------
// Point-partitioned problems (ba_set_exchange): the part of the problem's
// sums that this problem's observations contribute, laid out for one
// all-reduce each.
// ---------------------------------------------------------------------------

// out[c * os + i] = sum over camera c's pieces of part[. * PART + i], i < nv.
static __global__ void k_cam_sum_parts(int C, const int32_t* __restrict__ cam_piece_ptr,
                                       const double* __restrict__ part, int nv, int os, double* __restrict__ out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)C * nv) return;
  const int c = (int)(t / nv), i = (int)(t % nv);
  double sum = 0.0;
  for (int k = cam_piece_ptr[c]; k < cam_piece_ptr[c + 1]; ++k) sum += part[(long long)PART * k + i];
  out[(long long)os * c + i] = sum;
}

// The trial's sums over this part: out[0] cost (pieces), out[1] the model's
// quadratic term (pieces), out[2] gp . dp (chunks).
static __global__ void k_part_trial_sums(int npieces, const double* __restrict__ part, int npb,
                                         const double* __restrict__ dot_gp, double* __restrict__ out) {
  const double a = block_sum_array(part, npieces, PART);
  const double b = block_sum_array(part + 1, npieces, PART);
  const double c = block_sum_array(dot_gp, npb, 1);
  if (threadIdx.x == 0) {
    out[0] = a;
    out[1] = b;
    out[2] = c;
  }
}

// The cost over this part into out[0] (0 when gated off: F is not stale).
static __global__ void k_part_cost_sum(int npieces, const double* __restrict__ part, const DevState* st, int gate,
                                       double* __restrict__ out) {
  const bool skip = gate && !st->need_cost;
  const double F = skip ? 0.0 : block_sum_array(part, npieces, PART);
  if (threadIdx.x == 0) out[0] = F;
}

// st->F = the summed cost (when not gated off).
static __global__ void k_cost_set(DevState* st, int gate, const double* __restrict__ tot) {
  if (gate && !st->need_cost) return;
  st->F = tot[0];
  st->need_cost = 0;
  if (!isfinite(tot[0])) st->err |= 2;
}

// Sum the cost pieces into st->F (initial cost / after set_params).
static __global__ void k_cost_finalize(int npieces, const double* __restrict__ part, DevState* st, int gate) {
  if (gate && !st->need_cost) return;
  const double F = block_sum_array(part, npieces, PART);
  if (threadIdx.x == 0) {
    st->F = F;
    st->need_cost = 0;
    if (!isfinite(F)) st->err |= 2;
  }
}

// One LM decision: gain ratio rho = (F - Ft) / model with the model
// reduction -lin - quad / 2, accept iff Ft is finite, model > 0 and Ft < F,
// damping update; fills the stats record and returns the next damping.
__device__ __forceinline__ bool lm_decide(double F, double Ft, double quad, double lin, double lam, double pcg_rel,
                                          int pcg_iters, int fallbacks, double up, double down, double rho_good,
                                          double rho_bad, double lam_min, double lam_max, ba_iter_stats& sr,
                                          double& nl) {
  const double model = -lin - 0.5 * quad;
  const double rho = model != 0.0 ? (F - Ft) / model : nan("");
  const bool finite = isfinite(Ft);
  const bool accept = finite && model > 0.0 && Ft < F;
  sr.cost = F;
  sr.cost_trial = Ft;
  sr.model = model;
  sr.rho = rho;
  sr.lambda = lam;
  sr.pcg_rel_res = pcg_rel;
  sr.accepted = accept ? 1 : 0;
  sr.pcg_iters = pcg_iters;
  sr.precond_fallbacks = fallbacks;
  sr.reserved = 0;
  nl = lam;
  if (accept) {
    if (rho > rho_good) nl = fmax(lam / up, lam_min);
    else if (rho < rho_bad) nl = fmin(lam / down, lam_max);
  } else {
    nl = fmin(lam / down, lam_max);
  }
  return accept;
}

// Gain ratio, accept / reject and the damping update (one block).
// tot (a point-partitioned problem, else NULL): the trial cost, the model's
// quadratic term and gp . dp already summed over every part of the problem.
static __global__ void k_lm_control(int npieces, const double* __restrict__ part, int ncb,
                             const double* __restrict__ dot_gc, int npb, const double* __restrict__ dot_gp,
                             double up, double down, double rho_good, double rho_bad, double lam_min,
                             double lam_max, DevState* st, ba_iter_stats* __restrict__ stats, int cap,
                             const double* __restrict__ tot) {
  const double Ft = tot ? tot[0] : block_sum_array(part, npieces, PART);
  const double quad = tot ? tot[1] : block_sum_array(part + 1, npieces, PART);
  const double lin = block_sum_array(dot_gc, ncb, 1) + (tot ? tot[2] : block_sum_array(dot_gp, npb, 1));
  if (threadIdx.x != 0) return;
  const double F = st->F;
  const long long t = st->trials;
  double nl;
  const bool accept = lm_decide(F, Ft, quad, lin, st->lam, st->pcg_rel, st->pcg_iters, st->fallbacks, up, down,
                                rho_good, rho_bad, lam_min, lam_max, stats[t % cap], nl);
  if (!isfinite(Ft)) st->nonfinite += 1;
  if (accept) {
    st->cur = 1 - st->cur;
    st->F = Ft;
    st->need_lin = 1;
  } else {
    st->need_lin = 0;
  }
  st->lam = nl;
  st->trials = t + 1;
}

// ---------------------------------------------------------------------------
// Implicit-function adjoint (ba_backward)
// ---------------------------------------------------------------------------

// Right-hand side of H v = dL/dtheta in the forward solver's slots:
// gc = -dL/dcams, gp = -dL/dpoints (points to the internal numbering).
template <typename T>
static __global__ void k_adj_rhs(int C, int P, const T* __restrict__ dLc, const T* __restrict__ dLp,
                          const int32_t* __restrict__ pnew, double* __restrict__ gc, double* __restrict__ gp) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 9LL * C) gc[i] = dLc ? -(double)dLc[i] : 0.0;
  if (i < 3LL * P) {
    const long long j = i / 3, a = i % 3;
    gp[i] = dLp ? -(double)dLp[3LL * pnew[j] + a] : 0.0;
  }
}

// Camera-major pass over the pieces: e_k = sqrt(w) J_k v (v = (v_c, v_p)),
// dL/dx_k = sqrt(w) e_k written in input order, and per piece
// sum_k (sqrt(w) Jc_k)^T e_k = (H v)_c (J_l^T still to apply to the first
// three in the recompute mode).
template <typename T, bool MF>
static __global__ void __launch_bounds__(PIECE_THREADS)
k_adjoint_cam(const int32_t* __restrict__ piece_cam, const int32_t* __restrict__ piece_beg,
              const int32_t* __restrict__ piece_end, const int32_t* __restrict__ cm_pt,
              const int32_t* __restrict__ perm_cam, const T* __restrict__ cm_px, const T* __restrict__ Jcm,
              const T* __restrict__ cm_sw, const T* __restrict__ ptab, const T* __restrict__ camtab,
              const T* __restrict__ xv, const T* __restrict__ vp, T delta, int O, T* __restrict__ dpix,
              double* __restrict__ part) {
  __shared__ T sct[CT];
  __shared__ T sx[PV];
  const int b = blockIdx.x;
  const int c = piece_cam[b];
  constexpr int XS = pass_vec_stride(MF);
  if (threadIdx.x < CT) sct[threadIdx.x] = camtab[(long long)CT * c + threadIdx.x];
  if (threadIdx.x >= 32 && threadIdx.x < 32 + XS) sx[threadIdx.x - 32] = xv[(long long)XS * c + threadIdx.x - 32];
  __syncthreads();
  T acc[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) acc[i] = T(0);
  const int end = piece_end[b];
  for (int s = piece_beg[b] + threadIdx.x; s < end; s += PIECE_THREADS) {
    const int j = cm_pt[s];
    T X0, X1, X2, pad;
    load4(ptab + 8LL * j, X0, X1, X2, pad);
    // sqrt(w) from the residual at the current parameters
    T px, py, sc;
    project_obs(sct, X0, X1, X2, px, py, sc);
    const T r0 = sc * px - cm_px[s], r1 = sc * py - cm_px[(long long)O + s];
    T hr, w;
    const T sw = huber_weight(r0 * r0 + r1 * r1, delta, hr, w);
    const T d0 = vp[3LL * j], d1 = vp[3LL * j + 1], d2 = vp[3LL * j + 2];
    const T g0 = sct[0] * d0 + sct[1] * d1 + sct[2] * d2;
    const T g1 = sct[3] * d0 + sct[4] * d1 + sct[5] * d2;
    const T g2 = sct[6] * d0 + sct[7] * d1 + sct[8] * d2;
    T e0, e1;
    if (MF) {
      Fac<T> o;
      fac_obs(sct, X0, X1, X2, cm_sw ? cm_sw[s] : T(1), o);
      jc_times_fac(o, sx, e0, e1);
      e0 += o.A[0] * g0 + o.A[1] * g1 + o.A[2] * g2;
      e1 += o.A[3] * g0 + o.A[4] * g1 + o.A[5] * g2;
      jct_fac_acc(o, e0, e1, acc);
    } else {
      T pl[NPLANE];
      load_planes<NPLANE_JC>(Jcm, O, s, pl);
      T j0[9], j1[9];
      jc_rows(pl, j0, j1);
      e0 = pl[0] * g0 + pl[1] * g1 + pl[2] * g2;
      e1 = pl[3] * g0 + pl[4] * g1 + pl[5] * g2;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        e0 += j0[i] * sx[i];
        e1 += j1[i] * sx[i];
      }
#pragma unroll
      for (int i = 0; i < 9; ++i) acc[i] += j0[i] * e0 + j1[i] * e1;
    }
    const long long k = perm_cam[s];
    dpix[2 * k] = sw * e0;
    dpix[2 * k + 1] = sw * e1;
  }
  block_sum_store<9>(acc, part + (long long)PART * b);
}

// dL/dtheta0 for the cameras: a_c - (H* v)_c on frozen parameters, 0 on free
// ones (theta* does not depend on the start of the free parameters).
template <typename T, bool MF>
static __global__ void k_adjoint_combine(int C, const int32_t* __restrict__ cam_piece_ptr, const double* __restrict__ part,
                                  const double* __restrict__ U, const T* __restrict__ camtab,
                                  const double* __restrict__ lam_ptr, double dmin, double dmax,
                                  const double* __restrict__ vc, const T* __restrict__ dLc,
                                  const uint8_t* __restrict__ fixed, T* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double sum[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) sum[i] = 0.0;
  for (int k = cam_piece_ptr[c]; k < cam_piece_ptr[c + 1]; ++k)
#pragma unroll
    for (int i = 0; i < 9; ++i) sum[i] += part[(long long)PART * k + i];
  if (MF) {
    const T* Jl = camtab + (long long)CT * c + CT_JL;
    const double s0 = sum[0], s1 = sum[1], s2 = sum[2];
#pragma unroll
    for (int i = 0; i < 3; ++i) sum[i] = (double)Jl[i] * s0 + (double)Jl[3 + i] * s1 + (double)Jl[6 + i] * s2;
  }
  const double lam = *lam_ptr;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const double hv = sum[i] + damp(U[45LL * c + sym9(i, i)], lam, dmin, dmax) * vc[9LL * c + i];
    const bool fz = fixed && fixed[9LL * c + i];
    out[9LL * c + i] = fz ? (T)((dLc ? (double)dLc[9LL * c + i] : 0.0) - hv) : T(0);
  }
}

// ---------------------------------------------------------------------------
// Step-level helpers
// ---------------------------------------------------------------------------

// Camera vector (double [C][9]) to the pass form.
template <typename T, bool MF>
static __global__ void k_pass_vec(int C, const double* __restrict__ x, const T* __restrict__ camtab, T* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  write_pass_vec<T, MF>(camtab + (long long)CT * c, x + 9LL * c, out + (long long)pass_vec_stride(MF) * c);
}

// Unpack U [C][45] to [C][9][9] (or V [P][6] to [P][3][3]); block b of the
// output is packed block row[b] (row = NULL: b).
static __global__ void k_unpack_sym(long long n, int dim, const double* __restrict__ packed, const int32_t* __restrict__ row,
                             double* __restrict__ full) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * dim * dim) return;
  const long long ob = i / (dim * dim);
  const long long blk = row ? row[ob] : ob;
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

// Export sqrt(w) Jc [O][2][9], sqrt(w) Jp [O][2][3] and w [O] in input order,
// from the camera-major planes (stored mode) or recomputed exactly as the
// passes recompute them.
template <typename T, bool MF>
static __global__ void k_export_lin(int O, int P, const int32_t* __restrict__ perm_cam, const int32_t* __restrict__ ci,
                             const int32_t* __restrict__ cm_pt, const T* __restrict__ cm_px,
                             const T* __restrict__ Jcm, const T* __restrict__ cm_sw, const T* __restrict__ camtab,
                             const T* __restrict__ pts_buf, const DevState* __restrict__ st, T delta,
                             T* __restrict__ Jc, T* __restrict__ Jp, T* __restrict__ w) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= O) return;
  const long long k = perm_cam[s];
  const int c = ci[k];
  const T* ct = camtab + (long long)CT * c;
  T ctl[CT];
#pragma unroll
  for (int i = 0; i < CT; ++i) ctl[i] = ct[i];
  const T* pts = pts_buf + (long long)st->cur * 3 * P;
  const int j = cm_pt[s];
  T pl[NPLANE];
  cm_planes<T, MF>(Jcm, O, (int)s, ctl, pts, j, cm_sw, pl);
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
    jp_from(pl, ctl, jp);
#pragma unroll
    for (int i = 0; i < 6; ++i) Jp[6 * k + i] = jp[i];
  }
  if (w) {
    T px, py, sc;
    project_obs(ctl, pts[3LL * j], pts[3LL * j + 1], pts[3LL * j + 2], px, py, sc);
    const T r0 = sc * px - cm_px[s], r1 = sc * py - cm_px[(long long)O + s];
    T hr, ww;
    huber_weight(r0 * r0 + r1 * r1, delta, hr, ww);
    w[k] = ww;
  }
}

}  // namespace ba
