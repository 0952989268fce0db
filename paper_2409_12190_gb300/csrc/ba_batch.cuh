// Batched LM: many independent small problems in one persistent launch.
//
// The problems are concatenated into one problem object (disjoint cameras and
// points), so the symbolic phase keeps each problem's cameras, points,
// pieces and observation slots contiguous and in the order a problem of its
// own would have them.  One CTA of BT = PIECE_THREADS threads takes a whole
// problem at a time from a work list (longest first by default) and runs all
// of its LM trials (Alg. 1 with the Schur / block-Jacobi PCG solve of
// Sec. IV): the camera tables, U, g_c, the block-Jacobi inverses and the PCG
// vectors sit in shared memory, the per-observation and per-point arrays of
// the problem (a few hundred KB) stay in L2 across its PCG iterations, and
// the phases are separated by block barriers instead of kernel boundaries.
//
// Every sum is taken in the same order as in the single-problem kernels
// (same per-piece thread striding, same warp trees, warps in the same order,
// pieces and point chunks in the same order), and the per-observation and
// per-camera arithmetic is the same device code, so each problem's trial
// sequence is the one a problem of its own produces up to the fused
// multiply-adds the compiler forms in each kernel.  Within this kernel the
// result of a problem does not depend on the grid, the work order or the
// other problems.  No global atomics are used on the numeric path; the only
// atomic is the work-list counter.
#pragma once

#include <stddef.h>

#include "ba_kernels.cuh"

namespace ba {

constexpr int BT = PIECE_THREADS;  // threads per problem
constexpr int BMAXC = 28;          // cameras per problem: 9 * BMAXC <= BT
static_assert(9 * BMAXC <= BT, "the per-camera vector phase runs one thread per component");
static_assert(CHUNK_THREADS == BT, "point chunks are reduced with the block's threads");

// Per-problem LM state (device).
struct BState {
  double lam;        // damping of the next trial
  double F;          // cost at the current parameters
  long long trials;  // trials run so far
  int cur;           // parameter buffer holding theta
  int need_cost;     // F must be evaluated before the next trial
  int nonfinite;     // non-finite trial costs since the last stats read
  int err;           // bit 1: non-finite cost at the start
};

template <typename T>
struct BatchArgs {
  int nprob, C, P, O;  // totals
  const int32_t* cam_off;    // [nprob + 1] camera ranges
  const int32_t* pt_off;     // [nprob + 1] internal point ranges
  const int32_t* chunk_off;  // [nprob + 1] ranges of bchunk (nchunks + 1 entries per problem)
  const int32_t* bchunk;     // first point of each chunk of each problem, then its end
  const int32_t* order;      // [nprob] work list
  const int32_t* piece_cam;
  const int32_t* piece_beg;
  const int32_t* piece_end;
  const int32_t* cam_piece_ptr;
  const int32_t* cm_pt;
  const int32_t* rowptr_pt;
  const int32_t* pm2cm;
  const int32_t* pm_cam;
  const int32_t* pm_pt;
  const T* cm_px;
  const T* pm_px;
  T* cams;    // [2][C][9]
  T* pts;     // [2][P][3]
  T* camtab;  // [C][CT]
  T* ptab;    // [P][8]
  T* zbuf;    // [O][4]
  T* Jcm;     // stored mode planes or NULL
  T* cm_sw;   // sqrt(w), recompute mode under a robust loss, or NULL
  T* pm_sw;
  T* Vinv;
  T* y0;
  T* dp;
  double* V;
  double* gp;
  double* part;    // [npieces][PART]
  double* dot_gp;  // one per bchunk entry
  BState* state;
  ba_iter_stats* stats;  // [nprob][cap]
  int cap;
  int* work;
  int iters;
  T delta;
  double up, down, rho_good, rho_bad, lam_min, lam_max, dmin, dmax, tol;
  int maxiter;
};

// Shared memory of one CTA (one problem at a time).
template <typename T>
struct BShared {
  double U[BMAXC * 45];
  double M[BMAXC * 45];
  double gc[BMAXC * 9];
  double x[BMAXC * 9], r[BMAXC * 9], z[BMAXC * 9], p[BMAXC * 9], q[BMAXC * 9], ss[BMAXC * 9];
  double red[8 * 54];  // reduction scratch (float2 or double per slot)
  double tot[9];
  T ct[BMAXC][CT];  // camera tables of the linearisation
  T pT[BMAXC][PV];  // PCG direction in the passes' form
  T xT[BMAXC][PV];  // camera step in the passes' form
  double sce64[CT]; // camera table of the evaluated parameters (cost, in double)
  FFCam sceff;      // the same split into float-float pairs (FP32 cost)
  // recompute mode: padded copies of the camera tables and of the vector a
  // point-major pass reads (neighbouring slots use different cameras), and
  // the per-observation products of one point chunk
  T fct[BMAXC][17];
  T fxv[BMAXC][13];
  alignas(16) T sz[CHUNK_SLOTS * 4];  // read and written as 4-vectors
  double lam, F, rz_old, bb, pcg_rel, dot_gc;
  long long trials;
  int cur, need_lin, pcg_iters, fallbacks, widx;
};

static_assert(offsetof(BShared<float>, sz) % 16 == 0 && offsetof(BShared<double>, sz) % 16 == 0,
              "4-vector accesses to the chunk buffer need 16-byte alignment");

// ---------------------------------------------------------------------------
// Block reductions with the single-problem kernels' order (BT threads, 8
// warps; warp trees by shuffles, then the warps in order), on the CTA's
// scratch, each ending in a barrier so the scratch can be reused at once.
// ---------------------------------------------------------------------------

// = block_sum_store<NV, PRECISE> (float partials)
template <int NV, bool PRECISE>
__device__ __forceinline__ void bred_store(float (&v)[NV], double* scratch, double* __restrict__ out) {
  float2* red = reinterpret_cast<float2*>(scratch);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int nw = BT / 32;
  if constexpr (PRECISE && NV > 32 && NV <= 64) {
    float w[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) w[i] = i < NV ? v[i] : 0.f;
    float h0, l0, h1, l1;
    warp_rs64_ff(w, h0, l0, h1, l1);
    if (2 * lane < NV) red[warp * NV + 2 * lane] = make_float2(h0, l0);
    if (2 * lane + 1 < NV) red[warp * NV + 2 * lane + 1] = make_float2(h1, l1);
  } else if constexpr (!PRECISE && NV > 4 && NV <= 16) {
    float w[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) w[i] = i < NV ? v[i] : 0.f;
    const float s = warp_rs16_f(w);
    if ((lane & 1) == 0 && (lane >> 1) < NV) red[warp * NV + (lane >> 1)] = make_float2(s, 0.f);
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
    if (lane == 0) red[warp * NV + i] = make_float2(hi, lo);
  }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NV; i += BT) {
    float hi = red[i].x, lo = red[i].y;
    for (int w = 1; w < nw; ++w) {
      if (PRECISE) ff_add(hi, lo, red[w * NV + i].x, red[w * NV + i].y);
      else hi += red[w * NV + i].x;
    }
    out[i] = (double)hi + (double)lo;
  }
  __syncthreads();
}

// = block_sum_store<NV> (double partials)
template <int NV, bool PRECISE>
__device__ __forceinline__ void bred_store(double (&v)[NV], double* red, double* __restrict__ out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int nw = BT / 32;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const double s = warp_sum(v[i]);
    if (lane == 0) red[warp * NV + i] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NV; i += BT) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w * NV + i];
    out[i] = s;
  }
  __syncthreads();
}

// = block_sum_all<NV>: every thread gets the totals.
template <int NV, typename T>
__device__ __forceinline__ void bred_all(BShared<T>& S, double (&v)[NV]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int nw = BT / 32;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const double s = warp_sum(v[i]);
    if (lane == 0) S.red[warp * NV + i] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NV; i += BT) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += S.red[w * NV + i];
    S.tot[i] = s;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = S.tot[i];
  __syncthreads();
}

// = block_sum_array
template <typename T>
__device__ __forceinline__ double bred_array(BShared<T>& S, const double* __restrict__ a, int n, int stride) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += BT) s += a[(long long)i * stride];
  double v[1] = {s};
  bred_all<1>(S, v);
  return v[0];
}

// = block_sum_all over one warp of per-camera values (the 32-thread
// per-camera kernels): 0 + the warp tree.  Called by warp 0.
__device__ __forceinline__ double warp_total(double v) { return 0.0 + warp_sum(v); }

// ---------------------------------------------------------------------------
// Phases of one LM trial of problem b
// ---------------------------------------------------------------------------

template <typename T>
struct BRange {
  int c0, nc, j0, j1, q0, q1, k0, nk;
};

// Pass A, step 2 over the problem's point chunks: t_j (MODE 0) or the
// back-substitution (MODE 1, per-chunk partials of g_p . dp into dot_gp).
template <typename T, int MODE>
__device__ __forceinline__ void batch_pass_a2(const BatchArgs<T>& a, const BRange<T>& R, BShared<T>& S, int cur) {
  for (int kk = 0; kk < R.nk; ++kk) {
    const int js = a.bchunk[R.k0 + kk], je = a.bchunk[R.k0 + kk + 1];
    const int s0 = a.rowptr_pt[js], s1 = a.rowptr_pt[je];
    double gd = 0.0;
    if (s1 - s0 <= CHUNK_SLOTS) {
      for (int j = js + threadIdx.x; j < je; j += BT) {
        T z0 = 0, z1 = 0, z2 = 0;
        const int q1 = a.rowptr_pt[j + 1];
        for (int q = a.rowptr_pt[j]; q < q1; ++q) {
          const T* zz = a.zbuf + 4LL * a.pm2cm[q];
          z0 += zz[0];
          z1 += zz[1];
          z2 += zz[2];
        }
        gd += pass_a_point<T, MODE>(j, a.P, z0, z1, z2, a.Vinv, a.ptab, a.dp, a.y0, a.gp, a.pts, cur);
      }
    } else {
      T z0 = 0, z1 = 0, z2 = 0;
      for (int q = s0 + threadIdx.x; q < s1; q += BT) {
        T u0, u1, u2, u3;
        load4(a.zbuf + 4LL * a.pm2cm[q], u0, u1, u2, u3);
        z0 += u0;
        z1 += u1;
        z2 += u2;
      }
      double dd[3] = {(double)z0, (double)z1, (double)z2};
      bred_all<3>(S, dd);
      if (threadIdx.x == 0)
        gd = pass_a_point<T, MODE>(js, a.P, (T)dd[0], (T)dd[1], (T)dd[2], a.Vinv, a.ptab, a.dp, a.y0, a.gp, a.pts,
                                   cur);
    }
    if (MODE == 1) {
      double v[1] = {gd};
      bred_all<1>(S, v);
      if (threadIdx.x == 0) a.dot_gp[R.k0 + kk] = v[0];
    }
  }
}

// Pass A, step 1 over the problem's pieces with the camera vectors xv.
template <typename T, bool MF>
__device__ __forceinline__ void batch_pass_a1(const BatchArgs<T>& a, const BRange<T>& R, BShared<T>& S,
                                              T (*xv)[PV]) {
  for (int q = R.q0; q < R.q1; ++q) {
    const int c = a.piece_cam[q] - R.c0;
    T ctl[15], xl[9];
#pragma unroll
    for (int i = 0; i < 15; ++i) ctl[i] = S.ct[c][i];
#pragma unroll
    for (int i = 0; i < 9; ++i) xl[i] = xv[c][i];
    pass_a1_range<T, MF, BT>(a.piece_beg[q], a.piece_end[q], a.cm_pt, a.Jcm, a.cm_sw, a.ptab, ctl, xl, a.O, a.zbuf);
  }
}

// Point-major pass A of the recompute mode over the problem's point chunks
// (the cameras' padded tables and vectors in shared memory, the vector in
// S.fxv): z per observation into shared memory, then per point t_j
// (MODE 0, into the point table) or the back-substitution (MODE 1, with
// per-chunk partials of g_p . dp).  The same per-observation products and
// per-point sums as passes A1 + A2.
template <typename T, int MODE>
__device__ __forceinline__ void batch_pass_fa(const BatchArgs<T>& a, const BRange<T>& R, BShared<T>& S, int cur) {
  constexpr int U = CHUNK_SLOTS / BT;
  for (int kk = 0; kk < R.nk; ++kk) {
    const int js = a.bchunk[R.k0 + kk], je = a.bchunk[R.k0 + kk + 1];
    const int s0 = a.rowptr_pt[js], s1 = a.rowptr_pt[je];
    double gd = 0.0;
    if (s1 - s0 <= CHUNK_SLOTS) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int q = s0 + threadIdx.x + u * BT;
        if (q >= s1) continue;
        const int j = a.pm_pt[q];
        const int l = a.pm_cam[q] - R.c0;
        T X0, X1, X2, pad;
        load4(a.ptab + 8LL * j, X0, X1, X2, pad);
        T z0, z1, z2;
        a1_obs(&S.fct[l][0], &S.fxv[l][0], X0, X1, X2, a.pm_sw ? a.pm_sw[q] : T(1), z0, z1, z2);
        store4(S.sz + 4 * (q - s0), z0, z1, z2, T(0));
      }
      __syncthreads();
      for (int j = js + threadIdx.x; j < je; j += BT) {
        T z0 = 0, z1 = 0, z2 = 0;
        const int q1 = a.rowptr_pt[j + 1];
        for (int q = a.rowptr_pt[j]; q < q1; ++q) {
          z0 += S.sz[4 * (q - s0)];
          z1 += S.sz[4 * (q - s0) + 1];
          z2 += S.sz[4 * (q - s0) + 2];
        }
        gd += pass_a_point<T, MODE>(j, a.P, z0, z1, z2, a.Vinv, a.ptab, a.dp, a.y0, a.gp, a.pts, cur);
      }
      __syncthreads();
    } else {
      T z0 = 0, z1 = 0, z2 = 0;
      for (int q = s0 + threadIdx.x; q < s1; q += BT) {
        const int l = a.pm_cam[q] - R.c0;
        T X0, X1, X2, pad;
        load4(a.ptab + 8LL * a.pm_pt[q], X0, X1, X2, pad);
        T u0, u1, u2;
        a1_obs(&S.fct[l][0], &S.fxv[l][0], X0, X1, X2, a.pm_sw ? a.pm_sw[q] : T(1), u0, u1, u2);
        z0 += u0;
        z1 += u1;
        z2 += u2;
      }
      double dd[3] = {(double)z0, (double)z1, (double)z2};
      bred_all<3>(S, dd);
      if (threadIdx.x == 0)
        gd = pass_a_point<T, MODE>(js, a.P, (T)dd[0], (T)dd[1], (T)dd[2], a.Vinv, a.ptab, a.dp, a.y0, a.gp, a.pts,
                                   cur);
    }
    if (MODE == 1) {
      double v[1] = {gd};
      bred_all<1>(S, v);
      if (threadIdx.x == 0) a.dot_gp[R.k0 + kk] = v[0];
    }
  }
}

// Padded copy of camera vectors (the passes' form) for batch_pass_fa.
template <typename T>
__device__ __forceinline__ void batch_stage_fxv(BShared<T>& S, const BRange<T>& R, T (*xv)[PV]) {
  for (int i = threadIdx.x; i < R.nc * 9; i += BT) S.fxv[i / 9][i % 9] = xv[i / 9][i % 9];
  __syncthreads();
}

// The linearisation (a1 + a2) at the current parameters.
template <typename T, bool MF>
__device__ void batch_linearise(const BatchArgs<T>& a, const BRange<T>& R, BShared<T>& S, int cur) {
  const T* pts = a.pts + (long long)cur * 3 * a.P;
  if (threadIdx.x < R.nc) {
    const int c = R.c0 + threadIdx.x;
    camera_table(a.cams + (long long)cur * 9 * a.C + 9LL * c, S.ct[threadIdx.x]);
#pragma unroll
    for (int i = 0; i < CT; ++i) a.camtab[(long long)CT * c + i] = S.ct[threadIdx.x][i];
#pragma unroll
    for (int i = 0; i < 15; ++i) S.fct[threadIdx.x][i] = S.ct[threadIdx.x][i];
  }
  for (int j = R.j0 + threadIdx.x; j < R.j1; j += BT) {
    const T* X = pts + 3LL * j;
    store4(a.ptab + 8LL * j, X[0], X[1], X[2], T(0));
  }
  __syncthreads();
  for (int q = R.q0; q < R.q1; ++q) {
    const int c = a.piece_cam[q] - R.c0;
    T acc[54];
#pragma unroll
    for (int i = 0; i < 54; ++i) acc[i] = T(0);
    lin_cam_range<T, !MF, BT>(a.piece_beg[q], a.piece_end[q], a.cm_pt, a.cm_px, pts, S.ct[c], a.delta, a.O, a.Jcm,
                              a.cm_sw, acc);
    bred_store<54, true>(acc, S.red, a.part + (long long)PART * q);
  }
  if (threadIdx.x < R.nc) {
    const int c = R.c0 + threadIdx.x;
    cam_combine_lin_one(a.cam_piece_ptr[c], a.cam_piece_ptr[c + 1], a.part, S.U + 45 * threadIdx.x,
                        S.gc + 9 * threadIdx.x);
  }
  for (int kk = 0; kk < R.nk; ++kk) {
    const int js = a.bchunk[R.k0 + kk], je = a.bchunk[R.k0 + kk + 1];
    const int s0 = a.rowptr_pt[js], s1 = a.rowptr_pt[je];
    if (s1 - s0 <= CHUNK_SLOTS) {
      for (int j = js + threadIdx.x; j < je; j += BT) {
        T acc[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) acc[i] = T(0);
        const int q1 = a.rowptr_pt[j + 1];
        for (int q = a.rowptr_pt[j]; q < q1; ++q) {
          T v[9];
          lin_pt_obs<T>(q, a.O, a.pm_cam, a.pm_pt, a.pm_px, pts, a.camtab, a.delta, a.pm_sw, v);
#pragma unroll
          for (int i = 0; i < 9; ++i) acc[i] += v[i];
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) a.V[6LL * j + i] = (double)acc[i];
#pragma unroll
        for (int i = 0; i < 3; ++i) a.gp[3LL * j + i] = (double)acc[6 + i];
      }
    } else {
      T acc[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) acc[i] = T(0);
      for (int q = s0 + threadIdx.x; q < s1; q += BT) {
        T v[9];
        lin_pt_obs<T>(q, a.O, a.pm_cam, a.pm_pt, a.pm_px, pts, a.camtab, a.delta, a.pm_sw, v);
#pragma unroll
        for (int i = 0; i < 9; ++i) acc[i] += v[i];
      }
      double d[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) d[i] = (double)acc[i];
      bred_all<9>(S, d);
      if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < 6; ++i) a.V[6LL * js + i] = d[i];
#pragma unroll
        for (int i = 0; i < 3; ++i) a.gp[3LL * js + i] = d[6 + i];
      }
    }
  }
  __syncthreads();
}

// Cost 1/2 sum rho of the problem at parameter buffer buf (MODEL: with the
// quadratic model term at the linearisation, trial step in S.xT / a.dp);
// per-piece partials in a.part.
template <typename T, bool MODEL, bool MF>
__device__ void batch_cost(const BatchArgs<T>& a, const BRange<T>& R, BShared<T>& S, int buf, int cur) {
  const T* pts = a.pts + (long long)buf * 3 * a.P;
  const T* pts_old = a.pts + (long long)cur * 3 * a.P;
  for (int q = R.q0; q < R.q1; ++q) {
    const int cg = a.piece_cam[q];
    const int c = cg - R.c0;
    if (threadIdx.x == 0) {
      camera_table_f64(a.cams + (long long)buf * 9 * a.C + 9LL * cg, S.sce64);
      ffcam_from(S.sce64, S.sceff);
    }
    __syncthreads();
    double cost = 0.0, quad = 0.0;
    cost_cam_range<T, MODEL, MF, BT>(a.piece_beg[q], a.piece_end[q], a.cm_pt, a.cm_px, pts, pts_old, &S.sceff,
                                     S.sce64, S.ct[c], S.xT[c], a.delta, a.O, a.Jcm, a.cm_sw, a.dp, cost, quad);
    double v[2] = {cost, quad};
    bred_store<2, true>(v, S.red, a.part + (long long)PART * q);
  }
}

// One LM trial of the problem (Alg. 1): linearise if theta changed, damp,
// Schur complement and block-Jacobi PCG, back-substitution, trial cost and
// model reduction, accept / reject.
template <typename T, bool MF>
__device__ void batch_trial(const BatchArgs<T>& a, const BRange<T>& R, BShared<T>& S, int b) {
  const int tid = threadIdx.x;
  const int cur = S.cur;
  const double lam = S.lam;
  if (S.need_lin) batch_linearise<T, MF>(a, R, S, cur);

  // a3: damping, V*^{-1}, Schur pieces, block-Jacobi blocks
  for (int j = R.j0 + tid; j < R.j1; j += BT) pt_damp_one<T>(j, a.V, a.gp, lam, a.dmin, a.dmax, a.Vinv, a.y0);
  __syncthreads();
  {
    const T* pts = a.pts + (long long)cur * 3 * a.P;
    for (int q = R.q0; q < R.q1; ++q) {
      const int c = a.piece_cam[q] - R.c0;
      T acc[54];
#pragma unroll
      for (int i = 0; i < 54; ++i) acc[i] = T(0);
      schur_cam_range<T, MF, BT>(a.piece_beg[q], a.piece_end[q], a.cm_pt, a.Jcm, S.ct[c], pts, a.cm_sw, a.Vinv, a.y0,
                                 a.O, acc);
      bred_store<54, true>(acc, S.red, a.part + (long long)PART * q);
    }
  }
  if (tid < 32) {
    double rz = 0.0, bb = 0.0;
    int fb = 0;
    if (tid < R.nc) {
      const int cg = R.c0 + tid;
      cam_schur_one<T, MF, true>(a.cam_piece_ptr[cg], a.cam_piece_ptr[cg + 1], a.part, S.U + 45 * tid, S.gc + 9 * tid,
                           S.ct[tid], lam, a.dmin, a.dmax, nullptr, S.M + 45 * tid, S.x + 9 * tid, S.r + 9 * tid,
                           S.z + 9 * tid, S.p + 9 * tid, S.pT[tid], rz, bb, fb);
    }
    const int nfb = __popc(__ballot_sync(0xffffffffu, fb != 0));
    rz = warp_total(rz);
    bb = warp_total(bb);
    if (tid == 0) {
      S.rz_old = rz;
      S.bb = bb;
      S.fallbacks = nfb;
      S.pcg_iters = 0;
      S.pcg_rel = 1.0;
    }
  }
  __syncthreads();

  // a4: block-Jacobi PCG on S dc = b (thread lc*9 + i owns component i of
  // camera lc, as in the per-camera vector kernels)
  const int lc = tid / 9, ci = tid % 9;
  const bool ok = lc < R.nc;
  const int o = 9 * lc + ci;
  for (int k = 0; k < a.maxiter; ++k) {
    if (MF) {
      batch_stage_fxv(S, R, S.pT);
      batch_pass_fa<T, 0>(a, R, S, cur);
    } else {
      batch_pass_a1<T, MF>(a, R, S, S.pT);
      __syncthreads();
      batch_pass_a2<T, 0>(a, R, S, cur);
    }
    __syncthreads();
    for (int q = R.q0; q < R.q1; ++q) {
      const int c = a.piece_cam[q] - R.c0;
      T ctl[15];
#pragma unroll
      for (int i = 0; i < 15; ++i) ctl[i] = S.ct[c][i];
      T acc[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) acc[i] = T(0);
      // FP32 recompute mode: two gathers in flight per thread, next indices prefetched
      pass_b_range<T, MF, BT, (MF && sizeof(T) == 4) ? 2 : 1, (MF && sizeof(T) == 4)>(
          a.piece_beg[q], a.piece_end[q], a.cm_pt, a.Jcm, a.cm_sw, a.ptab, ctl, a.O, acc);
      bred_store<9, false>(acc, S.red, a.part + (long long)PART * q);
    }
    // q = U* p - (pass-B sums), p.q
    double pv = 0.0, sum = 0.0;
    if (ok) {
      pv = S.p[o];
      const int cg = R.c0 + lc;
      const int p1 = a.cam_piece_ptr[cg + 1];
      for (int kq = a.cam_piece_ptr[cg]; kq < p1; ++kq) sum += a.part[(long long)PART * kq + ci];
      S.ss[o] = sum;
    }
    __syncthreads();
    double pq = 0.0;
    if (ok) {
      if (MF && ci < 3) {
        const T* Jl = S.ct[lc] + CT_JL;
        sum = (double)Jl[ci] * S.ss[9 * lc] + (double)Jl[3 + ci] * S.ss[9 * lc + 1] +
              (double)Jl[6 + ci] * S.ss[9 * lc + 2];
      }
      const double* Uc = S.U + 45 * lc;
      double y = damp(Uc[sym9(ci, ci)], lam, a.dmin, a.dmax) * S.p[o];
#pragma unroll
      for (int j = 0; j < 9; ++j) y += Uc[sym9_rt(ci, j)] * S.p[9 * lc + j];
      y -= sum;
      S.q[o] = y;
      pq = pv * y;
    }
    {
      double v[1] = {pq};
      bred_all<1>(S, v);
      pq = v[0];
    }
    if (!(pq > 0.0) || !isfinite(pq)) {
      // no positive curvature (b = 0 or breakdown): keep x, stop
      if (tid == 0) {
        S.pcg_iters = k;
        if (k == 0) S.pcg_rel = 0.0;
      }
      break;
    }
    const double alpha = S.rz_old / pq;
    double rv = 0.0;
    if (ok) {
      S.x[o] += alpha * S.p[o];
      rv = S.r[o] - alpha * S.q[o];
      S.r[o] = rv;
    }
    __syncthreads();
    double zz = 0.0;
    if (ok) {
      const double* Mc = S.M + 45 * lc;
#pragma unroll
      for (int j = 0; j < 9; ++j) zz += Mc[sym9_rt(ci, j)] * S.r[9 * lc + j];
      S.z[o] = zz;
    }
    double v2[2] = {rv * zz, rv * rv};
    bred_all<2>(S, v2);
    const double rz_new = v2[0], rr = v2[1], rz_old = S.rz_old, bb = S.bb;
    const bool conv = sqrt(rr) <= a.tol * sqrt(bb);
    if (tid == 0) {
      S.pcg_iters = k + 1;
      S.pcg_rel = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    }
    if (conv) break;
    const double beta = rz_new / rz_old;
    if (ok) {
      const double pn = S.z[o] + beta * S.p[o];
      S.p[o] = pn;
    }
    __syncthreads();
    if (ok) {
      if (MF && ci < 3) {
        const T* Jl = S.ct[lc] + CT_JL;
        S.pT[lc][ci] = (T)((double)Jl[3 * ci] * S.p[9 * lc] + (double)Jl[3 * ci + 1] * S.p[9 * lc + 1] +
                           (double)Jl[3 * ci + 2] * S.p[9 * lc + 2]);
        S.pT[lc][9 + ci] = T(0);
      } else {
        S.pT[lc][ci] = (T)S.p[o];
      }
    }
    if (tid == 0) S.rz_old = rz_new;
    __syncthreads();
  }
  __syncthreads();

  // a5: trial cameras, back-substitution and trial points
  if (tid < 32) {
    double gd = 0.0;
    if (tid < R.nc) {
      const int cg = R.c0 + tid;
      gd = cam_trial_one<T, MF>(S.x + 9 * tid, S.gc + 9 * tid, a.cams + (long long)cur * 9 * a.C + 9LL * cg,
                                a.cams + (long long)(1 - cur) * 9 * a.C + 9LL * cg, S.ct[tid], S.xT[tid]);
    }
    gd = warp_total(gd);
    if (tid == 0) S.dot_gc = gd;
  }
  __syncthreads();
  if (MF) {
    batch_stage_fxv(S, R, S.xT);
    batch_pass_fa<T, 1>(a, R, S, cur);
  } else {
    batch_pass_a1<T, MF>(a, R, S, S.xT);
    __syncthreads();
    batch_pass_a2<T, 1>(a, R, S, cur);
  }
  __syncthreads();

  // a6: trial cost, model reduction, accept / reject
  batch_cost<T, true, MF>(a, R, S, 1 - cur, cur);
  const double Ft = bred_array(S, a.part + (long long)PART * R.q0, R.q1 - R.q0, PART);
  const double quad = bred_array(S, a.part + (long long)PART * R.q0 + 1, R.q1 - R.q0, PART);
  const double lin = bred_array(S, &S.dot_gc, 1, 1) + bred_array(S, a.dot_gp + R.k0, R.nk, 1);
  if (tid == 0) {
    const long long t = S.trials;
    double nl;
    const bool accept = lm_decide(S.F, Ft, quad, lin, lam, S.pcg_rel, S.pcg_iters, S.fallbacks, a.up, a.down,
                                  a.rho_good, a.rho_bad, a.lam_min, a.lam_max,
                                  a.stats[(long long)b * a.cap + t % a.cap], nl);
    if (!isfinite(Ft)) a.state[b].nonfinite += 1;
    if (accept) {
      S.cur = 1 - cur;
      S.F = Ft;
      S.need_lin = 1;
    } else {
      S.need_lin = 0;
    }
    S.lam = nl;
    S.trials = t + 1;
  }
  __syncthreads();
}

// All trials of problem b.
template <typename T, bool MF>
__device__ void batch_problem(const BatchArgs<T>& a, int b, BShared<T>& S) {
  BRange<T> R;
  R.c0 = a.cam_off[b];
  R.nc = a.cam_off[b + 1] - R.c0;
  R.j0 = a.pt_off[b];
  R.j1 = a.pt_off[b + 1];
  R.q0 = a.cam_piece_ptr[R.c0];
  R.q1 = a.cam_piece_ptr[R.c0 + R.nc];
  R.k0 = a.chunk_off[b];
  R.nk = a.chunk_off[b + 1] - R.k0 - 1;
  if (threadIdx.x == 0) {
    const BState st = a.state[b];
    S.lam = st.lam;
    S.F = st.F;
    S.trials = st.trials;
    S.cur = st.cur;
    // the linearisation is a function of theta alone: rebuild it for each
    // launch instead of keeping U and g_c across launches
    S.need_lin = 1;
  }
  __syncthreads();
  if (a.state[b].need_cost) {
    const int cur = S.cur;
    batch_cost<T, false, MF>(a, R, S, cur, cur);
    const double F = bred_array(S, a.part + (long long)PART * R.q0, R.q1 - R.q0, PART);
    if (threadIdx.x == 0) {
      S.F = F;
      a.state[b].need_cost = 0;
      if (!isfinite(F)) a.state[b].err |= 2;
    }
    __syncthreads();
  }
  for (int it = 0; it < a.iters; ++it) batch_trial<T, MF>(a, R, S, b);
  if (threadIdx.x == 0) {
    BState& st = a.state[b];
    st.lam = S.lam;
    st.F = S.F;
    st.trials = S.trials;
    st.cur = S.cur;
  }
  __syncthreads();
}

// The persistent kernel: CTAs take problems from the work list until it is
// empty.  MINB is the CTAs per SM the register allocation is bounded for.
template <typename T, bool MF, int MINB>
static __global__ void __launch_bounds__(BT, MINB) k_batch_lm(BatchArgs<T> a) {
  extern __shared__ __align__(16) unsigned char braw[];
  BShared<T>& S = *reinterpret_cast<BShared<T>*>(braw);
  for (;;) {
    if (threadIdx.x == 0) S.widx = atomicAdd(a.work, 1);
    __syncthreads();
    const int w = S.widx;
    __syncthreads();
    if (w >= a.nprob) break;
    batch_problem<T, MF>(a, a.order[w], S);
  }
}

// Global problem-local indices -> indices of the concatenated problem
// (out-of-range local indices become -1, which the symbolic phase rejects).
static __global__ void k_batch_globalize(int O, int nprob, const int32_t* __restrict__ obs_off,
                                  const int32_t* __restrict__ cam_off, const int32_t* __restrict__ pt_off,
                                  const int32_t* __restrict__ ci, const int32_t* __restrict__ pi,
                                  int32_t* __restrict__ gci, int32_t* __restrict__ gpi) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= O) return;
  int lo = 0, hi = nprob;  // obs_off[lo] <= k < obs_off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (obs_off[mid] <= k) lo = mid;
    else hi = mid;
  }
  const int c = ci[k], p = pi[k];
  const int nc = cam_off[lo + 1] - cam_off[lo], np = pt_off[lo + 1] - pt_off[lo];
  gci[k] = (c >= 0 && c < nc) ? cam_off[lo] + c : -1;
  gpi[k] = (p >= 0 && p < np) ? pt_off[lo] + p : -1;
}

// Current parameters of every problem in the caller's order.
template <typename T>
static __global__ void k_batch_params(int nprob, int C, int P, const int32_t* __restrict__ cam_off,
                               const int32_t* __restrict__ pt_off, const int32_t* __restrict__ pnewpos,
                               const BState* __restrict__ state, const T* __restrict__ cams,
                               const T* __restrict__ pts, T* __restrict__ cams_out, T* __restrict__ pts_out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cams_out && i < C) {
    int lo = 0, hi = nprob;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (cam_off[mid] <= i) lo = mid;
      else hi = mid;
    }
    const T* src = cams + (long long)state[lo].cur * 9 * C + 9 * i;
#pragma unroll
    for (int k = 0; k < 9; ++k) cams_out[9 * i + k] = src[k];
  }
  if (pts_out && i < P) {
    const int j = pnewpos[i];  // internal index of the caller's point i
    int lo = 0, hi = nprob;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (pt_off[mid] <= j) lo = mid;
      else hi = mid;
    }
    const T* src = pts + (long long)state[lo].cur * 3 * P + 3LL * j;
#pragma unroll
    for (int k = 0; k < 3; ++k) pts_out[3 * i + k] = src[k];
  }
}

}  // namespace ba
