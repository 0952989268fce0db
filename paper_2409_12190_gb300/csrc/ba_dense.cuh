// Direct solve of the reduced camera system (the paper's sparse direct
// solver, Sec. IV-C, "Sparse Direct Solver (Cholesky Factorization)"; here
// the reduced system S = U* - W V*^{-1} W^T is formed explicitly as a dense
// n x n matrix, n = 9C, and factored by a blocked Cholesky in FP64).
//
//   k_schur_dense    one CTA per camera i builds block row i of S:
//                    -sum over the points j of camera i, over the
//                    observations l of j, of W_k V*_j^{-1} W_l^T into block
//                    (i, camera(l)), then + U*_i on the diagonal block.  The
//                    camera's observations are taken one at a time (the
//                    targets of one point's observations are distinct
//                    cameras, so they are updated in parallel without
//                    conflict) and in slot order: every entry is a fixed-
//                    order sum, bitwise reproducible, no atomics.
//   k_dense_mask     S -> m S m + (I - m) for frozen parameters.
//   k_chol_diag      factor the diagonal DB x DB block of the current block
//                    column (one CTA, in shared memory).
//   k_chol_panel     L_ik = A_ik L_kk^{-T} for the block rows below (one
//                    warp per block of rows).
//   k_chol_update    A_IJ -= L_Ik L_Jk^T on the trailing lower triangle.
//   k_dense_solve    L L^T x = b (one CTA: forward then backward
//                    substitution, column by column), x into the PCG
//                    solution vector; a failed factorisation (a pivot not
//                    positive or not finite) gives x = 0 and is counted.
// The matrix is row-major with leading dimension n; only its lower triangle
// is referenced after the build.
#pragma once

#include "ba_kernels.cuh"

namespace ba {

constexpr int DB = 32;             // Cholesky block size
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
              int O, const T* __restrict__ Vinv, const double* __restrict__ U, const double* __restrict__ lam_ptr,
              double dmin, double dmax, double* __restrict__ S) {
  __shared__ T spl[DENSE_MAXQ + 1][NPLANE];  // planes of the staged observations (last: observation k)
  __shared__ double sY[27];                  // W_k V*^{-1}
  __shared__ double sW[DENSE_MAXQ][27];      // W_l of the staged observations
  __shared__ int sq[DENSE_MAXQ];             // their cameras
  const int i = blockIdx.x;
  const long long n = 9LL * C;
  const int tid = threadIdx.x;
  // zero block row i
  double* row = S + 9LL * i * n;
  for (long long e = tid; e < 9 * n; e += DENSE_THREADS) row[e] = 0.0;
  const T* pts = pts_buf + (long long)st->cur * 3 * P;
  const T* cti = camtab + (long long)CT * i;
  const int s0 = rowptr_cam[i], s1 = rowptr_cam[i + 1];
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
  // + U*_i on the diagonal block
  if (tid < 81) {
    const int a = tid / 9, b = tid % 9;
    const double* Ui = U + 45LL * i;
    double u = Ui[a <= b ? sym9(a, b) : sym9(b, a)];
    if (a == b) u += damp(u, *lam_ptr, dmin, dmax);
    row[(long long)a * n + 9LL * i + b] += u;
  }
}

// S -> m S m + (I - m) for frozen camera parameters (fixed [C][9], nonzero =
// frozen).
static __global__ void k_dense_mask(long long n, const uint8_t* __restrict__ fixed, double* __restrict__ S) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const long long r = e / n, c = e % n;
  if (fixed[r] || fixed[c]) S[e] = (r == c) ? 1.0 : 0.0;
}

// Factor the diagonal block at (k, k), k = kb * DB, of size nb = min(DB, n - k).
static __global__ void __launch_bounds__(DB * DB / 4)
k_chol_diag(int n, int kb, double* __restrict__ A, int* __restrict__ fail) {
  __shared__ double L[DB][DB + 1];
  const int k = kb * DB;
  const int nb = min(DB, n - k);
  const int tid = threadIdx.x;
  for (int e = tid; e < DB * DB; e += blockDim.x) {
    const int r = e / DB, c = e % DB;
    L[r][c] = (r < nb && c < nb) ? A[(long long)(k + r) * n + k + c] : 0.0;
  }
  __syncthreads();
  for (int c = 0; c < nb; ++c) {
    // the pivot's reciprocal square root: one FP64 sequence on the
    // column's critical path, then multiplications (a division per entry
    // and a square root cost as much each on this GPU's FP64 pipe)
    const double d = L[c][c];
    const bool ok = d > 0.0 && isfinite(d);
    const double rs = ok ? rsqrt(d) : 1.0;
    __syncthreads();
    if (tid == 0) {
      L[c][c] = ok ? d * rs : 1.0;
      if (!ok) *fail = 1;
    }
    // column below the pivot
    for (int r = c + 1 + tid; r < nb; r += blockDim.x) L[r][c] *= rs;
    __syncthreads();
    // rank-1 update of the trailing lower triangle (its m (m + 1) / 2 entries)
    const int m = nb - c - 1;
    for (int e = tid; e < m * (m + 1) / 2; e += blockDim.x) {
      int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);  // FP32 guess, corrected below
      while ((r + 1) * (r + 2) / 2 <= e) ++r;
      while (r * (r + 1) / 2 > e) --r;
      const int cc = e - r * (r + 1) / 2;  // 0 <= cc <= r
      L[c + 1 + r][c + 1 + cc] -= L[c + 1 + r][c] * L[c + 1 + cc][c];
    }
    __syncthreads();
  }
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int r = e / nb, c = e % nb;
    if (c <= r) A[(long long)(k + r) * n + k + c] = L[r][c];
  }
}

// L_ik = A_ik L_kk^{-T} for the block rows below block column kb; one CTA
// per block of DB rows, one thread per row solving its DB unknowns.
static __global__ void __launch_bounds__(DB)
k_chol_panel(int n, int kb, double* __restrict__ A) {
  __shared__ double Lk[DB][DB + 1];
  const int k = kb * DB;
  const int nb = min(DB, n - k);
  const int r0 = k + nb + blockIdx.x * DB;
  const int tid = threadIdx.x;
  for (int c = 0; c < nb; ++c) Lk[tid][c] = tid < nb ? A[(long long)(k + tid) * n + k + c] : 0.0;
  __syncthreads();
  const int r = r0 + tid;
  if (r >= n) return;
  double x[DB];
#pragma unroll
  for (int c = 0; c < DB; ++c) x[c] = c < nb ? A[(long long)r * n + k + c] : 0.0;
  // x L_kk^T = a: x_c = (a_c - sum_{m<c} x_m L_cm) / L_cc
#pragma unroll
  for (int c = 0; c < DB; ++c) {
    if (c < nb) {
      double v = x[c];
#pragma unroll
      for (int m = 0; m < c; ++m) v -= x[m] * Lk[c][m];
      x[c] = v / Lk[c][c];
    }
  }
#pragma unroll
  for (int c = 0; c < DB; ++c)
    if (c < nb) A[(long long)r * n + k + c] = x[c];
}

// A_IJ -= L_Ik L_Jk^T for the trailing tiles I >= J (DB x DB each) below
// block column kb; blockIdx.x enumerates the lower-triangular tiles.
static __global__ void __launch_bounds__(DB * DB / 4)
k_chol_update(int n, int kb, double* __restrict__ A) {
  __shared__ double LI[DB][DB + 1], LJ[DB][DB + 1];
  const int k = kb * DB;
  const int t0 = kb + 1;  // first trailing block
  // tile (I, J), I >= J >= 0 relative to t0, from the triangular index
  const long long t = blockIdx.x;
  int I = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((long long)(I + 1) * (I + 2) / 2 <= t) ++I;
  while ((long long)I * (I + 1) / 2 > t) --I;
  const int J = (int)(t - (long long)I * (I + 1) / 2);
  const int rI = (t0 + I) * DB, rJ = (t0 + J) * DB;
  const int tid = threadIdx.x;
  for (int e = tid; e < DB * DB; e += blockDim.x) {
    const int r = e / DB, c = e % DB;
    LI[r][c] = (rI + r < n) ? A[(long long)(rI + r) * n + k + c] : 0.0;
    LJ[r][c] = (rJ + r < n) ? A[(long long)(rJ + r) * n + k + c] : 0.0;
  }
  __syncthreads();
  // 4 entries per thread: rows r, r + 8, r + 16, r + 24 of column c
  const int c = tid % DB, rb = tid / DB;
  for (int rr = rb; rr < DB; rr += (DB * DB / 4) / DB) {
    const int gr = rI + rr, gc = rJ + c;
    if (gr >= n || gc >= n || gc > gr) continue;
    double v = 0.0;
#pragma unroll
    for (int m = 0; m < DB; ++m) v += LI[rr][m] * LJ[c][m];
    A[(long long)gr * n + gc] -= v;
  }
}

// x = (L L^T)^{-1} b (b = r, the reduced right-hand side); one CTA, by
// blocks of DB unknowns: solve a block's DB x DB triangle (one warp, column
// by column, with the reciprocals of its diagonal), then update every
// remaining right-hand-side entry with the block (coalesced rows of L).  bw: the half-bandwidth of L (L_ij = 0 for
// i - j > bw; n - 1 for a dense matrix), which bounds those updates.  With a
// failed factorisation x = 0 (the LM trial is then a rejection) and the
// failure is counted in st->fallbacks.  Writes the solve's statistics.
static __global__ void __launch_bounds__(1024)
k_dense_solve(int n, int bw, const double* __restrict__ L, const double* __restrict__ b, double* __restrict__ y,
              double* __restrict__ x, const int* __restrict__ fail, DevState* st) {
  __shared__ double sb[DB];
  __shared__ double tl[DB][DB + 1];  // the diagonal block's triangle
  __shared__ double ri[DB];          // reciprocals of its diagonal
  const int tid = threadIdx.x;
  const int lane = tid % 32;
  const bool bad = *fail != 0;
  for (int i = tid; i < n; i += blockDim.x) y[i] = bad ? 0.0 : b[i];
  __syncthreads();
  const int nblk = (n + DB - 1) / DB;
  // stage block kb's triangle and the reciprocals of its diagonal
  auto stage = [&](int k, int nb) {
    for (int e = tid; e < DB * DB; e += blockDim.x) {
      const int rr = e / DB, cc = e % DB;
      tl[rr][cc] = (rr < nb && cc <= rr) ? L[(long long)(k + rr) * n + k + cc] : 0.0;
    }
    __syncthreads();
    if (tid < nb) ri[tid] = 1.0 / tl[tid][tid];
    __syncthreads();
  };
  if (!bad) {
    // forward: L y = b.  A block's triangle is solved column by column by
    // warp 0 (lane r holds y_r; y_c = y_c / L_cc, then every lane r > c
    // subtracts L_rc y_c)
    for (int kb = 0; kb < nblk; ++kb) {
      const int k = kb * DB, nb = min(DB, n - k);
      stage(k, nb);
      if (tid < 32) {
        double v = lane < nb ? y[k + lane] : 0.0;
        for (int c = 0; c < nb; ++c) {
          const double yc = __shfl_sync(0xffffffffu, v * ri[c], c);
          if (lane > c) v -= tl[lane][c] * yc;
          if (lane == c) v = yc;
        }
        if (lane < nb) {
          sb[lane] = v;
          y[k + lane] = v;
        }
      }
      __syncthreads();
      const int iend = min(n, k + nb + bw);
      for (int i = k + nb + tid; i < iend; i += blockDim.x) {
        double v = 0.0;
        for (int c = 0; c < nb; ++c) v += L[(long long)i * n + k + c] * sb[c];
        y[i] -= v;
      }
      __syncthreads();
    }
    // backward: L^T x = y (column by column from the last: x_c = y_c / L_cc,
    // then every lane r < c subtracts L_cr x_c)
    for (int kb = nblk - 1; kb >= 0; --kb) {
      const int k = kb * DB, nb = min(DB, n - k);
      stage(k, nb);
      if (tid < 32) {
        double v = lane < nb ? y[k + lane] : 0.0;
        for (int c = nb - 1; c >= 0; --c) {
          const double xc = __shfl_sync(0xffffffffu, v * ri[c], c);
          if (lane < c) v -= tl[c][lane] * xc;
          if (lane == c) v = xc;
        }
        if (lane < nb) {
          sb[lane] = v;
          y[k + lane] = v;
        }
      }
      __syncthreads();
      for (int i = max(0, k - bw) + tid; i < k; i += blockDim.x) {
        double v = 0.0;
        for (int c = 0; c < nb; ++c) v += L[(long long)(k + c) * n + i] * sb[c];
        y[i] -= v;
      }
      __syncthreads();
    }
  }
  for (int i = tid; i < n; i += blockDim.x) x[i] = y[i];
  if (tid == 0) {
    st->pcg_done = 1;
    st->pcg_iters = 0;
    st->pcg_rel = bad ? 1.0 : 0.0;
    if (bad) st->fallbacks += 1;
  }
}

}  // namespace ba
