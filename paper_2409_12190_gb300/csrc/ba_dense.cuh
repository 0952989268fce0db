// Direct solve of the reduced camera system (the paper's sparse direct
// solver, Sec. IV-C, "Sparse Direct Solver (Cholesky Factorization)"; here
// the reduced system S = U* - W V*^{-1} W^T is formed explicitly as a dense
// n x n matrix, n = 9C, and factored in FP64 by the band-tile task graph of
// ba_band.cuh with the band the whole lower triangle).
//
//   k_schur_dense    nseg CTAs per camera i build nseg partial block rows of
//                    S: each takes a contiguous share of camera i's
//                    observations in slot order and, for each (point j),
//                    subtracts W_k V*_j^{-1} W_l^T over the observations l of
//                    j from block (i, camera(l)).  The targets of one point's
//                    observations are distinct cameras, so they are updated
//                    in parallel without conflict: every partial entry is a
//                    fixed-order sum, no atomics.
//   k_schur_to_band  S = U* + the partials summed in segment order, frozen
//                    parameters as identity rows and columns, into the band
//                    tiles (lower triangle).
#pragma once

#include "ba_kernels.cuh"

namespace ba {

constexpr int DB = 32;             // Cholesky tile size
constexpr int DENSE_THREADS = 256;
constexpr int DENSE_MAXQ = 16;     // observations of one point staged at a time

// Entry e = 3 a + m of W = Jc^T Jp (9 x 3, row a of Jc^T, column m of Jp)
// from an observation's planes, in double.
template <typename T>
__device__ __forceinline__ double w_entry(const T* __restrict__ pl, int e) {
  T j0[9], j1[9];
  jc_rows(pl, j0, j1);
  const int a = e / 3, m = e % 3;
  return (double)j0[a] * (double)pl[NPLANE_JC + m] + (double)j1[a] * (double)pl[NPLANE_JC + 3 + m];
}

template <typename T, bool MF>
static __global__ void __launch_bounds__(DENSE_THREADS)
k_schur_dense(int C, const int32_t* __restrict__ rowptr_cam, const int32_t* __restrict__ cm_pt,
              const int32_t* __restrict__ rowptr_pt, const int32_t* __restrict__ pm_cam,
              const int32_t* __restrict__ pm2cm, const T* __restrict__ Jcm, const T* __restrict__ cm_sw,
              const T* __restrict__ camtab, const T* __restrict__ pts_buf, const DevState* __restrict__ st, int P,
              int O, const T* __restrict__ Vinv, int nseg, double* __restrict__ Spart) {
  __shared__ T spl[DENSE_MAXQ + 1][NPLANE];  // planes of the staged observations (last: observation k)
  __shared__ double sY[27];                  // W_k V*^{-1}
  __shared__ double sW[DENSE_MAXQ][27];      // W_l of the staged observations
  __shared__ int sq[DENSE_MAXQ];             // their cameras
  const int i = blockIdx.x / nseg, seg = blockIdx.x % nseg;
  const long long n = 9LL * C;
  const int tid = threadIdx.x;
  // zero this segment's partial block row i
  double* row = Spart + (long long)seg * n * n + 9LL * i * n;
  for (long long e = tid; e < 9 * n; e += DENSE_THREADS) row[e] = 0.0;
  const T* pts = pts_buf + (long long)st->cur * 3 * P;
  const T* cti = camtab + (long long)CT * i;
  const int sa = rowptr_cam[i], sb = rowptr_cam[i + 1], per = (sb - sa + nseg - 1) / nseg;
  const int s0 = min(sb, sa + seg * per), s1 = min(sb, s0 + per);
  __syncthreads();
  for (int s = s0; s < s1; ++s) {
    const int j = cm_pt[s];
    // Y = W_k V*_j^{-1}
    if (tid == 0) {
      T pl[NPLANE];
      cm_planes<T, MF>(Jcm, O, s, cti, pts, j, cm_sw, pl);
#pragma unroll
      for (int p = 0; p < NPLANE; ++p) spl[DENSE_MAXQ][p] = pl[p];
    }
    __syncthreads();
    double y = 0.0;
    if (tid < 27) {
      const int a = tid / 3, m = tid % 3;
      const T* vi = Vinv + 6LL * j;
      const double v0 = (double)vi[m == 0 ? 0 : (m == 1 ? 1 : 2)];
      const double v1 = (double)vi[m == 0 ? 1 : (m == 1 ? 3 : 4)];
      const double v2 = (double)vi[m == 0 ? 2 : (m == 1 ? 4 : 5)];
      y = w_entry(spl[DENSE_MAXQ], 3 * a) * v0 + w_entry(spl[DENSE_MAXQ], 3 * a + 1) * v1 +
          w_entry(spl[DENSE_MAXQ], 3 * a + 2) * v2;
    }
    if (tid < 27) sY[tid] = y;
    const int q0 = rowptr_pt[j], q1 = rowptr_pt[j + 1];
    for (int qb = q0; qb < q1; qb += DENSE_MAXQ) {
      const int nq = min(DENSE_MAXQ, q1 - qb);
      // planes of up to DENSE_MAXQ observations of point j, one thread each
      if (tid < nq) {
        const int q = qb + tid;
        const int c2 = pm_cam[q];
        T pl[NPLANE];
        cm_planes<T, MF>(Jcm, O, pm2cm[q], camtab + (long long)CT * c2, pts, j, cm_sw, pl);
#pragma unroll
        for (int p = 0; p < NPLANE; ++p) spl[tid][p] = pl[p];
        sq[tid] = c2;
      }
      __syncthreads();
      for (int t = tid; t < nq * 27; t += DENSE_THREADS) sW[t / 27][t % 27] = w_entry(spl[t / 27], t % 27);
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
