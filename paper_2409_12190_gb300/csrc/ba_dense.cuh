// Direct solve of the reduced camera system (the paper's sparse direct
// solver, Sec. IV-C, "Sparse Direct Solver (Cholesky Factorization)"; here
// the reduced system S = U* - W V*^{-1} W^T is formed explicitly as a dense
// n x n matrix, n = 9C, and factored in FP64 by the band-tile task graph of
// ba_band.cuh with the band the whole lower triangle).
//
//   k_dense_w        W_k = Jc_k^T Jp_k of every observation, once per trial.
//   k_schur_dense    one CTA per (camera i, segment) builds a partial block
//                    row of S: for each observation k of its share of camera
//                    i's observations (slot order) it subtracts
//                    W_k V*_j^{-1} W_l^T from block (i, camera(l)) over the
//                    observations l of k's point j.  The CTA owns its
//                    partial row: every entry is a fixed-order sum, no
//                    atomics.
//   k_schur_to_band  S = U* + the partials summed in segment order, frozen
//                    parameters as identity rows and columns, into the band
//                    tiles (lower triangle).
#pragma once

#include "ba_kernels.cuh"

namespace ba {

constexpr int DB = 32;             // Cholesky tile size
constexpr int DENSE_THREADS = 256;
constexpr int DENSE_MAXQ = 16;     // observations of one point staged at a time

// W_k = Jc_k^T Jp_k (9 x 3, row-major, in double) of every observation, at
// its camera-major slot: one thread per point, over its observations.
template <typename T, bool MF>
static __global__ void __launch_bounds__(DENSE_THREADS)
k_dense_w(int P, const int32_t* __restrict__ rowptr_pt, const int32_t* __restrict__ pm_cam,
          const int32_t* __restrict__ pm2cm, const T* __restrict__ Jcm, const T* __restrict__ cm_sw,
          const T* __restrict__ camtab, const T* __restrict__ pts_buf, const DevState* __restrict__ st, int O,
          double* __restrict__ W) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P) return;
  const T* pts = pts_buf + (long long)st->cur * 3 * P;
  for (int q = rowptr_pt[j]; q < rowptr_pt[j + 1]; ++q) {
    const int s = pm2cm[q];
    T pl[NPLANE];
    cm_planes<T, MF>(Jcm, O, s, camtab + (long long)CT * pm_cam[q], pts, j, cm_sw, pl);
    T j0[9], j1[9];
    jc_rows(pl, j0, j1);
    double* w = W + 27LL * s;
#pragma unroll
    for (int a = 0; a < 9; ++a)
#pragma unroll
      for (int m = 0; m < 3; ++m)
        w[3 * a + m] = (double)j0[a] * (double)pl[NPLANE_JC + m] + (double)j1[a] * (double)pl[NPLANE_JC + 3 + m];
  }
}

// Partial block rows of -W V*^{-1} W^T: one CTA per (camera i, segment),
// the segment a contiguous share of camera i's observations in slot order.
// For each observation k (point j): Y = W_k V*_j^{-1} (27 threads); then, a
// chunk of at most DENSE_MAXQ observations l of j at a time, their W_l are
// staged and block (i, camera(l)) -= Y W_l^T over the chunk's 81 nq
// entries.  The targets of one point's observations are distinct cameras,
// so a chunk's updates do not conflict; the CTA owns its partial row, and
// every entry is a fixed-order sum, no atomics.
template <typename T>
static __global__ void __launch_bounds__(DENSE_THREADS)
k_schur_dense(int C, int nseg, const int32_t* __restrict__ rowptr_cam, const int32_t* __restrict__ cm_pt,
              const int32_t* __restrict__ rowptr_pt, const int32_t* __restrict__ pm_cam,
              const int32_t* __restrict__ pm2cm, const double* __restrict__ W, const T* __restrict__ Vinv,
              double* __restrict__ Spart) {
  __shared__ double sY[27];                  // W_k V*^{-1}
  __shared__ double sW[DENSE_MAXQ][27];      // W_l of the staged observations
  __shared__ int sq[DENSE_MAXQ];             // their cameras
  const int i = blockIdx.x / nseg, seg = blockIdx.x % nseg;
  const long long n = 9LL * C;
  const int tid = threadIdx.x;
  double* row = Spart + (long long)seg * n * n + 9LL * i * n;
  for (long long e = tid; e < 9 * n; e += DENSE_THREADS) row[e] = 0.0;
  const int sa = rowptr_cam[i], sb = rowptr_cam[i + 1], per = (sb - sa + nseg - 1) / nseg;
  const int s0 = min(sb, sa + seg * per), s1 = min(sb, s0 + per);
  __syncthreads();
  for (int s = s0; s < s1; ++s) {
    const int j = cm_pt[s];
    if (tid < 27) {
      // column m of V*_j^{-1} (packed upper: 00 01 02 11 12 22)
      const int a = tid / 3, m = tid % 3;
      const T* vi = Vinv + 6LL * j;
      const double v0 = (double)vi[m == 0 ? 0 : (m == 1 ? 1 : 2)];
      const double v1 = (double)vi[m == 0 ? 1 : (m == 1 ? 3 : 4)];
      const double v2 = (double)vi[m == 0 ? 2 : (m == 1 ? 4 : 5)];
      const double* wk = W + 27LL * s + 3 * a;
      sY[tid] = wk[0] * v0 + wk[1] * v1 + wk[2] * v2;
    }
    const int q0 = rowptr_pt[j], q1 = rowptr_pt[j + 1];
    for (int qb = q0; qb < q1; qb += DENSE_MAXQ) {
      const int nq = min(DENSE_MAXQ, q1 - qb);
      for (int t = tid; t < nq * 27; t += DENSE_THREADS) sW[t / 27][t % 27] = W[27LL * pm2cm[qb + t / 27] + t % 27];
      if (tid < nq) sq[tid] = pm_cam[qb + tid];
      __syncthreads();
      // S[9i + a][9 c2 + b] -= sum_m Y[a][m] W_l[b][m]
      for (int t = tid; t < nq * 81; t += DENSE_THREADS) {
        const int u = t / 81, ab = t % 81, a = ab / 9, b = ab % 9;
        const double d = sY[3 * a] * sW[u][3 * b] + sY[3 * a + 1] * sW[u][3 * b + 1] + sY[3 * a + 2] * sW[u][3 * b + 2];
        row[(long long)a * n + 9LL * sq[u] + b] -= d;
      }
      __syncthreads();
    }
  }
}

// S = U* + sum over the nseg partials (in segment order) for the lower
// triangle, rows and columns of frozen parameters (fixed [C][9], nonzero =
// frozen) replaced by the identity, into the band tiles T (tile size DB,
// tile (I, J) at (J (bwt + 1) + I - J) DB^2); one CTA per row r.
static __global__ void k_schur_to_band(int C, int nseg, const double* __restrict__ Spart,
                                       const double* __restrict__ U, const double* __restrict__ lam_ptr,
                                       double dmin, double dmax, const uint8_t* __restrict__ fixed, int bwt,
                                       double* __restrict__ T) {
  const long long n = 9LL * C;
  const int r = blockIdx.x;
  const int ci = r / 9, a = r % 9;
  const bool fr = fixed && fixed[r];
  for (int c = threadIdx.x; c <= r; c += blockDim.x) {
    double v = 0.0;
    for (int k = 0; k < nseg; ++k) v += Spart[(long long)k * n * n + (long long)r * n + c];
    if (c / 9 == ci) {
      const int b = c % 9;
      double u = U[45LL * ci + (a <= b ? sym9(a, b) : sym9(b, a))];
      if (a == b) u += damp(u, *lam_ptr, dmin, dmax);
      v += u;
    }
    if (fr || (fixed && fixed[c])) v = (r == c) ? 1.0 : 0.0;
    const int I = r / DB, J = c / DB;
    T[((long long)J * (bwt + 1) + (I - J)) * (DB * DB) + (r % DB) * DB + c % DB] = v;
  }
}

}  // namespace ba
