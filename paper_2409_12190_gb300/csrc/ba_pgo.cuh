// Pose-graph optimisation (Sec. IV-D, Eqs. 3-4): the paper's second
// problem, run by the same LM loop (Alg. 1) as bundle adjustment.
//
//   F(Z) = 1/2 sum_e r_e^T Omega_e r_e,   r_e = Log(zeta_i^{-1} zeta_j T_e^{-1})
//
// Tangent vectors are (rho, phi), translation first; an update is the left
// retraction zeta <- Exp(delta) zeta.  With E = zeta_i^{-1} zeta_j T_e^{-1}
// and A = J_l(r)^{-1} Ad(zeta_i^{-1}), dr/d(delta_j) = A = -dr/d(delta_i),
// so every edge contributes the one symmetric block B_e = A^T Omega A:
//
//   H_ii = sum_{e at i} B_e,   (H x)_i = sum_{e at i} B_e (x_i - x_other(e)),
//   g_i  = sum_{e at i} (+-) A^T Omega r_e   (- at the edge's first node).
//
// Everything is FP64.  Poses are stored as 8 doubles (t[3], q[4] = (x, y, z,
// w), pad), unit quaternions.
//
//   k_pgo_lin        per edge: r, A, B (full 6 x 6), q = A^T Omega r
//   k_pgo_node       per node: H_ii and g_i, fixed-order sums over the
//                    node's incident edges (CSR of the 2E incidences)
//   k_pgo_damp       per node: damping lambda clamp(diag H_ii), the
//                    block-Jacobi inverse (H_ii + D_i)^{-1}, b = -g
//   k_pgo_pcg        the whole PCG in one cooperative launch (bounded grid
//                    barriers, two per iteration)
//   k_pgo_trial      per node: zeta_i' = Exp(delta_i) zeta_i, g . delta
//   k_pgo_edge_cost  per edge: 1/2 r^T Omega r at the trial (or current)
//                    poses and 1/2 u^T B u, u = delta_j - delta_i
//   k_pgo_control    the gain ratio and the LM decision (shared rule)
//   k_pgo_band       block row i of H + D into the band tiles of the Cholesky
//                    solver (ba_band.cuh)
#pragma once

#include <cuda/atomic>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ba_band.cuh"
#include "ba_kernels.cuh"

namespace ba {

constexpr int PGO_NODE_THREADS = 128;
constexpr int PGO_EDGE_THREADS = 128;
// PCG: 6 threads per node (one per row), 32 nodes per block pass
constexpr int PGO_PCG_THREADS = 192;
constexpr int PGO_PCG_NODES = PGO_PCG_THREADS / 6;

// ---------------------------------------------------------------------------
// SO(3) / SE(3) in FP64
// ---------------------------------------------------------------------------

struct Pose {
  double t[3];
  double q[4];  // x, y, z, w
};

__device__ __forceinline__ Pose load_pose(const double* __restrict__ p) {
  const double4_32a a = *reinterpret_cast<const double4_32a*>(p);
  const double4_32a b = *reinterpret_cast<const double4_32a*>(p + 4);
  Pose o;
  o.t[0] = a.x;
  o.t[1] = a.y;
  o.t[2] = a.z;
  o.q[0] = a.w;
  o.q[1] = b.x;
  o.q[2] = b.y;
  o.q[3] = b.z;
  return o;
}

__device__ __forceinline__ void store_pose(double* __restrict__ p, const Pose& o) {
  *reinterpret_cast<double4_32a*>(p) = make_double4_32a(o.t[0], o.t[1], o.t[2], o.q[0]);
  *reinterpret_cast<double4_32a*>(p + 4) = make_double4_32a(o.q[1], o.q[2], o.q[3], 0.0);
}

// Rotation matrix of a unit quaternion (row-major).
__device__ __forceinline__ void quat_rot(const double* q, double* R) {
  const double x = q[0], y = q[1], z = q[2], w = q[3];
  R[0] = 1.0 - 2.0 * (y * y + z * z);
  R[1] = 2.0 * (x * y - z * w);
  R[2] = 2.0 * (x * z + y * w);
  R[3] = 2.0 * (x * y + z * w);
  R[4] = 1.0 - 2.0 * (x * x + z * z);
  R[5] = 2.0 * (y * z - x * w);
  R[6] = 2.0 * (x * z - y * w);
  R[7] = 2.0 * (y * z + x * w);
  R[8] = 1.0 - 2.0 * (x * x + y * y);
}

// Hamilton product a * b.
__device__ __forceinline__ void quat_mul(const double* a, const double* b, double* o) {
  o[0] = a[3] * b[0] + a[0] * b[3] + a[1] * b[2] - a[2] * b[1];
  o[1] = a[3] * b[1] - a[0] * b[2] + a[1] * b[3] + a[2] * b[0];
  o[2] = a[3] * b[2] + a[0] * b[1] - a[1] * b[0] + a[2] * b[3];
  o[3] = a[3] * b[3] - a[0] * b[0] - a[1] * b[1] - a[2] * b[2];
}

__device__ __forceinline__ void quat_normalise(double* q) {
  const double n = rsqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  const double s = q[3] < 0.0 ? -n : n;
  for (int k = 0; k < 4; ++k) q[k] *= s;
}

__device__ __forceinline__ void mat3_vec(const double* M, const double* v, double* o) {
  for (int i = 0; i < 3; ++i) o[i] = M[3 * i] * v[0] + M[3 * i + 1] * v[1] + M[3 * i + 2] * v[2];
}

__device__ __forceinline__ void mat3T_vec(const double* M, const double* v, double* o) {
  for (int i = 0; i < 3; ++i) o[i] = M[i] * v[0] + M[3 + i] * v[1] + M[6 + i] * v[2];
}

__device__ __forceinline__ void mat3_mul(const double* A, const double* B, double* C) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

__device__ __forceinline__ void skew3(const double* v, double* K) {
  K[0] = 0.0;
  K[1] = -v[2];
  K[2] = v[1];
  K[3] = v[2];
  K[4] = 0.0;
  K[5] = -v[0];
  K[6] = -v[1];
  K[7] = v[0];
  K[8] = 0.0;
}

// E = zeta_i^{-1} zeta_j T^{-1} as (q_E, t_E):
//   T_j T^{-1} = (R_j R_m^T, t_j - R_j R_m^T t_m),
//   zeta_i^{-1} X = (R_i^T R_X, R_i^T (t_X - t_i)).
__device__ __forceinline__ void edge_error(const Pose& Pi, const Pose& Pj, const Pose& Pm, double* qE, double* tE) {
  const double qmc[4] = {-Pm.q[0], -Pm.q[1], -Pm.q[2], Pm.q[3]};
  const double qic[4] = {-Pi.q[0], -Pi.q[1], -Pi.q[2], Pi.q[3]};
  double qjm[4];
  quat_mul(Pj.q, qmc, qjm);
  quat_mul(qic, qjm, qE);
  double Rjm[9], Ri[9], v[3];
  quat_rot(qjm, Rjm);
  mat3_vec(Rjm, Pm.t, v);
  quat_rot(Pi.q, Ri);
  const double d[3] = {Pj.t[0] - v[0] - Pi.t[0], Pj.t[1] - v[1] - Pi.t[1], Pj.t[2] - v[2] - Pi.t[2]};
  mat3T_vec(Ri, d, tE);
}

// Coefficients of the SE(3) left Jacobian and its inverse at rotation angle
// th (series below th = 0.1, each truncated after its t^6 term):
//   c1 = (th - sin th)/th^3, c2 = (th^2 + 2 cos th - 2)/(2 th^4),
//   c3 = (2 th - 3 sin th + th cos th)/(2 th^5),
//   ci = (1 - (th/2) cot(th/2)) / th^2.
__device__ __forceinline__ void se3_coeffs(double th, double& c1, double& c2, double& c3, double& ci) {
  const double t2 = th * th;
  if (th < 0.1) {
    c1 = 1.0 / 6.0 - t2 * (1.0 / 120.0 - t2 * (1.0 / 5040.0 - t2 / 362880.0));
    c2 = 1.0 / 24.0 - t2 * (1.0 / 720.0 - t2 * (1.0 / 40320.0 - t2 / 3628800.0));
    c3 = 1.0 / 120.0 - t2 * (1.0 / 2520.0 - t2 * (1.0 / 120960.0 - t2 / 9979200.0));
    ci = 1.0 / 12.0 + t2 * (1.0 / 720.0 + t2 * (1.0 / 30240.0 + t2 / 1209600.0));
  } else {
    const double s = sin(th), c = cos(th);
    c1 = (th - s) / (t2 * th);
    c2 = (t2 + 2.0 * c - 2.0) / (2.0 * t2 * t2);
    c3 = (2.0 * th - 3.0 * s + th * c) / (2.0 * t2 * t2 * th);
    const double h = 0.5 * th;
    ci = (1.0 - h * cos(h) / sin(h)) / t2;
  }
}

// Log of (q, t): phi = 2 atan2(|v|, w) v/|v| (w >= 0; series of atan(x)/x
// below |v| < 1e-4 w), rho = J_l(phi)^{-1} t with
// J_l^{-1} = I - phi^/2 + ci phi^2.  Also returns |phi|.
__device__ __forceinline__ double se3_log(const double* q_in, const double* t, double* xi) {
  double q[4] = {q_in[0], q_in[1], q_in[2], q_in[3]};
  if (q[3] < 0.0)
    for (int k = 0; k < 4; ++k) q[k] = -q[k];
  const double s = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
  double f;
  if (s < 1e-4 * q[3]) {
    const double x2 = (s / q[3]) * (s / q[3]);
    f = 2.0 / q[3] * (1.0 - x2 * (1.0 / 3.0 - x2 / 5.0));
  } else {
    f = 2.0 * atan2(s, q[3]) / s;
  }
  const double phi[3] = {f * q[0], f * q[1], f * q[2]};
  const double th = sqrt(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]);
  double c1, c2, c3, ci;
  se3_coeffs(th, c1, c2, c3, ci);
  // J^{-1} t = t - (phi x t)/2 + ci (phi (phi . t) - th^2 t)
  const double pt = phi[0] * t[0] + phi[1] * t[1] + phi[2] * t[2];
  const double cx[3] = {phi[1] * t[2] - phi[2] * t[1], phi[2] * t[0] - phi[0] * t[2], phi[0] * t[1] - phi[1] * t[0]};
  for (int k = 0; k < 3; ++k) {
    xi[k] = t[k] - 0.5 * cx[k] + ci * (phi[k] * pt - th * th * t[k]);
    xi[3 + k] = phi[k];
  }
  return th;
}

// J_l(xi)^{-1} (6 x 6, row-major) = [[P, -P Q P], [0, P]], P = J_l(phi)^{-1}
// and Q(rho, phi) the upper-right block of the SE(3) left Jacobian:
//   Q = rho^/2 + c1 (phi^ rho^ + rho^ phi^ + phi^ rho^ phi^)
//       + c2 (phi^ phi^ rho^ + rho^ phi^ phi^ - 3 phi^ rho^ phi^)
//       + c3 (phi^ rho^ phi^ phi^ + phi^ phi^ rho^ phi^).
__device__ __forceinline__ void se3_jlinv(const double* xi, double th, double* Ji) {
  double c1, c2, c3, ci;
  se3_coeffs(th, c1, c2, c3, ci);
  double Pk[9], Rk[9];
  skew3(xi + 3, Pk);
  skew3(xi, Rk);
  double PR[9], RP[9], PP[9], PRP[9], PPR[9], RPP[9], PRPP[9], PPRP[9];
  mat3_mul(Pk, Rk, PR);
  mat3_mul(Rk, Pk, RP);
  mat3_mul(Pk, Pk, PP);
  mat3_mul(PR, Pk, PRP);
  mat3_mul(PP, Rk, PPR);
  mat3_mul(RP, Pk, RPP);
  mat3_mul(PRP, Pk, PRPP);
  mat3_mul(Pk, PRP, PPRP);
  double Q[9], P[9];
  for (int k = 0; k < 9; ++k) {
    Q[k] = 0.5 * Rk[k] + c1 * (PR[k] + RP[k] + PRP[k]) + c2 * (PPR[k] + RPP[k] - 3.0 * PRP[k]) +
           c3 * (PRPP[k] + PPRP[k]);
    P[k] = (k % 4 == 0 ? 1.0 : 0.0) - 0.5 * Pk[k] + ci * PP[k];
  }
  double QP[9], M[9];
  mat3_mul(Q, P, QP);
  mat3_mul(P, QP, M);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      Ji[6 * i + j] = P[3 * i + j];
      Ji[6 * i + 3 + j] = -M[3 * i + j];
      Ji[6 * (3 + i) + j] = 0.0;
      Ji[6 * (3 + i) + 3 + j] = P[3 * i + j];
    }
}

// Residual r = Log(E) and A = J_l(r)^{-1} Ad(zeta_i^{-1}), with
// Ad(zeta_i^{-1}) = [[R_i^T, -R_i^T t_i^], [0, R_i^T]].
__device__ __forceinline__ void edge_linear(const Pose& Pi, const Pose& Pj, const Pose& Pm, double* r, double* A) {
  double qE[4], tE[3];
  edge_error(Pi, Pj, Pm, qE, tE);
  const double th = se3_log(qE, tE, r);
  double Ji[36];
  se3_jlinv(r, th, Ji);
  double Ri[9], Tk[9];
  quat_rot(Pi.q, Ri);
  skew3(Pi.t, Tk);
  double RtT[9];  // R_i^T t_i^
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) RtT[3 * i + j] = Ri[i] * Tk[j] + Ri[3 + i] * Tk[3 + j] + Ri[6 + i] * Tk[6 + j];
  double Ad[36];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      Ad[6 * i + j] = Ri[3 * j + i];
      Ad[6 * i + 3 + j] = -RtT[3 * i + j];
      Ad[6 * (3 + i) + j] = 0.0;
      Ad[6 * (3 + i) + 3 + j] = Ri[3 * j + i];
    }
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double s = 0.0;
      for (int k = 0; k < 6; ++k) s += Ji[6 * i + k] * Ad[6 * k + j];
      A[6 * i + j] = s;
    }
}

__device__ __forceinline__ void load_info(const double* __restrict__ u, double* Om) {
  int k = 0;
  for (int a = 0; a < 6; ++a)
    for (int b = a; b < 6; ++b) {
      Om[6 * a + b] = u[k];
      Om[6 * b + a] = u[k];
      ++k;
    }
}

// Exp(delta) zeta: R' = R(phi) R, t' = R(phi) t + J_l(phi) rho; the
// quaternion of R(phi) is (sin(th/2)/th phi, cos(th/2)) (series of
// sin(th/2)/th below th = 1e-3).
__device__ __forceinline__ Pose retract(const Pose& P, const double* d) {
  double R[9], Jl[9];
  so3_tables(d[3], d[4], d[5], R, Jl);
  const double th = sqrt(d[3] * d[3] + d[4] * d[4] + d[5] * d[5]);
  double sh, ch;
  if (th < 1e-3) {
    const double t2 = th * th;
    sh = 0.5 - t2 * (1.0 / 48.0 - t2 / 3840.0);
    ch = cos(0.5 * th);
  } else {
    sh = sin(0.5 * th) / th;
    ch = cos(0.5 * th);
  }
  const double qd[4] = {sh * d[3], sh * d[4], sh * d[5], ch};
  Pose o;
  quat_mul(qd, P.q, o.q);
  quat_normalise(o.q);
  double Rt[3], Jr[3];
  mat3_vec(R, P.t, Rt);
  mat3_vec(Jl, d, Jr);
  for (int k = 0; k < 3; ++k) o.t[k] = Rt[k] + Jr[k];
  return o;
}

// ---------------------------------------------------------------------------
// Device state of the LM loop: ba's DevState (lam, F, cur, need_lin, PCG
// statistics, trial count) is reused as is.
// ---------------------------------------------------------------------------

// Per edge: r, A, B = A^T Omega A (full), q = A^T Omega r.  Skipped when the
// poses did not change since the last linearisation (st->need_lin == 0).
static __global__ void __launch_bounds__(PGO_EDGE_THREADS)
k_pgo_lin(int E, const int32_t* __restrict__ ei, const int32_t* __restrict__ ej, const double* __restrict__ meas,
          const double* __restrict__ info, const double* __restrict__ poses_buf, int N, const DevState* st,
          int force, double* __restrict__ B, double* __restrict__ qv, double* __restrict__ r_out,
          double* __restrict__ A_out) {
  if (!force && !st->need_lin) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const double* poses = poses_buf + (long long)st->cur * 8 * N;
  const Pose Pi = load_pose(poses + 8LL * ei[e]);
  const Pose Pj = load_pose(poses + 8LL * ej[e]);
  const Pose Pm = load_pose(meas + 8LL * e);
  double r[6], A[36], Om[36];
  edge_linear(Pi, Pj, Pm, r, A);
  load_info(info + 21LL * e, Om);
  double OA[36], Or[6];
  for (int a = 0; a < 6; ++a) {
    double s = 0.0;
    for (int k = 0; k < 6; ++k) s += Om[6 * a + k] * r[k];
    Or[a] = s;
    for (int b = 0; b < 6; ++b) {
      double t = 0.0;
      for (int k = 0; k < 6; ++k) t += Om[6 * a + k] * A[6 * k + b];
      OA[6 * a + b] = t;
    }
  }
  double* Be = B + 36LL * e;
  for (int a = 0; a < 6; ++a) {
    double s = 0.0;
    for (int k = 0; k < 6; ++k) s += A[6 * k + a] * Or[k];
    qv[6LL * e + a] = s;
    for (int b = a; b < 6; ++b) {
      double t = 0.0;
      for (int k = 0; k < 6; ++k) t += A[6 * k + a] * OA[6 * k + b];
      Be[6 * a + b] = t;
      Be[6 * b + a] = t;
    }
  }
  if (r_out)
    for (int a = 0; a < 6; ++a) r_out[6LL * e + a] = r[a];
  if (A_out)
    for (int a = 0; a < 36; ++a) A_out[36LL * e + a] = A[a];
}

// Per node: H_ii = sum B_e (upper triangle, 21) and g_i = sum (+-) q_e over
// the node's incidences in CSR order (inc = 2 e for the edge's first node,
// 2 e + 1 for its second).
static __global__ void __launch_bounds__(PGO_NODE_THREADS)
k_pgo_node(int N, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ inc, const double* __restrict__ B,
           const double* __restrict__ qv, const DevState* st, int force, double* __restrict__ Hd,
           double* __restrict__ g) {
  if (!force && !st->need_lin) return;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  double h[21], gg[6];
  for (int k = 0; k < 21; ++k) h[k] = 0.0;
  for (int k = 0; k < 6; ++k) gg[k] = 0.0;
  const int end = rowptr[n + 1];
  for (int s = rowptr[n]; s < end; ++s) {
    const int code = inc[s];
    const int e = code >> 1;
    const double sg = (code & 1) ? 1.0 : -1.0;
    const double* Be = B + 36LL * e;
    int k = 0;
    for (int a = 0; a < 6; ++a)
      for (int b = a; b < 6; ++b) h[k++] += Be[6 * a + b];
    for (int a = 0; a < 6; ++a) gg[a] += sg * qv[6LL * e + a];
  }
  for (int k = 0; k < 21; ++k) Hd[21LL * n + k] = h[k];
  for (int a = 0; a < 6; ++a) g[6LL * n + a] = gg[a];
}

__host__ __device__ constexpr int sym6(int a, int b) { return 6 * a - (a * (a - 1)) / 2 + (b - a); }

// Per node: D_i = lambda clamp(diag H_ii), M_i = (H_ii + D_i)^{-1} (full,
// by Cholesky; 0 for a fixed node or a block that is not SPD, counted),
// b_i = -g_i (0 for a fixed node), the PCG start x = 0, r = b, and the
// block partial of |b|^2.  Clears st->need_lin for the next trial.
static __global__ void __launch_bounds__(PGO_NODE_THREADS)
k_pgo_damp(int N, const double* __restrict__ Hd, const double* __restrict__ g, const uint8_t* __restrict__ fixed,
           const double* __restrict__ lam_ptr, double dmin, double dmax, double* __restrict__ D,
           double* __restrict__ Minv, double* __restrict__ x, double* __restrict__ r, double* __restrict__ part,
           DevState* st) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const double lam = *lam_ptr;
  double bb = 0.0;
  int bad = 0;
  if (n < N) {
    const bool fx = fixed && fixed[n];
    const double* h = Hd + 21LL * n;
    double L[6][6];
    double d[6];
    for (int a = 0; a < 6; ++a) d[a] = fx ? 0.0 : lam * fmin(fmax(h[sym6(a, a)], dmin), dmax);
    bool ok = !fx;
    for (int j = 0; j < 6 && ok; ++j) {
      double s = h[sym6(j, j)] + d[j];
      for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
      if (!(s > 0.0) || !isfinite(s)) {
        ok = false;
        break;
      }
      L[j][j] = sqrt(s);
      for (int i = j + 1; i < 6; ++i) {
        double t = h[sym6(j, i)];
        for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
        L[i][j] = t / L[j][j];
      }
    }
    double Mi[36];
    if (ok) {
      // M = L^{-T} L^{-1}: invert L column by column
      double Li[6][6];
      for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) Li[i][j] = 0.0;
      for (int j = 0; j < 6; ++j) {
        Li[j][j] = 1.0 / L[j][j];
        for (int i = j + 1; i < 6; ++i) {
          double s = 0.0;
          for (int k = j; k < i; ++k) s -= L[i][k] * Li[k][j];
          Li[i][j] = s / L[i][i];
        }
      }
      for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) {
          double s = 0.0;
          for (int k = (a > b ? a : b); k < 6; ++k) s += Li[k][a] * Li[k][b];
          Mi[6 * a + b] = s;
        }
    } else {
      for (int k = 0; k < 36; ++k) Mi[k] = 0.0;
      if (!fx) bad = 1;
    }
    for (int k = 0; k < 36; ++k) Minv[36LL * n + k] = Mi[k];
    for (int a = 0; a < 6; ++a) {
      const double b = fx ? 0.0 : -g[6LL * n + a];
      D[6LL * n + a] = d[a];
      x[6LL * n + a] = 0.0;
      r[6LL * n + a] = b;
      bb += b * b;
    }
  }
  double v[2] = {bb, (double)bad};
  block_sum_store<2>(v, part + 2LL * blockIdx.x);
  if (blockIdx.x == 0 && threadIdx.x == 0) st->need_lin = 0;
}

// ---------------------------------------------------------------------------
// PCG in one cooperative launch
// ---------------------------------------------------------------------------

struct GridBar {
  unsigned int count;
  unsigned int gen;
  int err;  // set by a barrier wait that ran out; every later wait returns
};

// Bounded grid-wide barrier (all blocks co-resident: cooperative launch).
// Thread 0 of each block arrives with an acquire-release increment of the
// counter (its block's writes, ordered before it by the block barrier, are
// released with it); the last block to arrive resets the counter and
// releases the next generation, which the others poll with acquire loads.
// Returns false if the wait ran out or another block's did (gb->err).
__device__ __forceinline__ bool grid_barrier(GridBar* gb, unsigned int nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> cnt(gb->count), gen(gb->gen);
    cuda::atomic_ref<int, cuda::thread_scope_device> err(gb->err);
    const unsigned int g0 = gen.load(cuda::memory_order_relaxed);
    const unsigned int arrived = cnt.fetch_add(1u, cuda::memory_order_acq_rel);
    int ok = 1;
    if (arrived == nblocks - 1) {
      cnt.store(0u, cuda::memory_order_relaxed);
      gen.fetch_add(1u, cuda::memory_order_release);
    } else {
      // 2^25 polls (all but the first 256 after a >= 32 ns sleep): a
      // second or more before giving up
      unsigned int spins = 0;
      while (gen.load(cuda::memory_order_acquire) == g0) {
        if (err.load(cuda::memory_order_relaxed) || ++spins > (1u << 25)) {
          ok = 0;
          err.store(1, cuda::memory_order_relaxed);
          break;
        }
        if (spins > 256) __nanosleep(32);
      }
    }
    s_ok = ok && !err.load(cuda::memory_order_relaxed);
  }
  __syncthreads();
  return s_ok != 0;
}

// Fixed-order sum of part[0..n) (NV interleaved values per entry), the same
// in every block.
template <int NV>
__device__ __forceinline__ void grid_total(const double* __restrict__ part, int n, double (&out)[NV]) {
  for (int k = 0; k < NV; ++k) out[k] = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    for (int k = 0; k < NV; ++k) out[k] += __ldcg(part + (long long)NV * i + k);
  block_sum_all<NV>(out);
}

struct PcgArgs {
  int N;
  int npb;             // nodes per block pass (blockDim.x = 6 npb)
  const int32_t* rowptr;
  const int2* inc2;    // per incidence slot: (edge, other node)
  const double* B;
  const double* D;
  const double* Minv;
  const uint8_t* fixed;
  double* x;
  double* r;
  double* z;
  double* p;  // [2][6N]: the direction of the previous and this iteration
  double* q;
  double* part;      // [grid][4]
  const double* bpart;  // |b|^2 partials of k_pgo_damp, [nbp][2]
  int nbp;
  int maxiter;
  double tol;
  GridBar* bar;
  DevState* st;
};

// Slots of neighbour directions staged in shared memory per pass.
constexpr int PGO_PCG_STAGE = 256;

// Block-Jacobi PCG on (H + D) x = b from x = 0, the iteration of the
// oracle's pcg: stop after the first iteration with |r| <= tol |b|, after
// maxiter, or (before updating x) when p^T (H + D) p is not positive.
// A block takes npb consecutive nodes per pass, thread (node, row).  Two
// grid barriers per iteration: the direction p = z + beta p_old of a
// neighbour is formed on the fly from its z and p_old (both complete at the
// last barrier).  The product first stages the neighbours' directions of
// the block's incidence slots in shared memory (every load independent),
// then each row sums B_e row . (p_i - p_other) over its node's slots in CSR
// order.  Read-only arrays go through the non-coherent cache; arrays the
// kernel writes are read from L2 (__ldcg).
static __global__ void __launch_bounds__(PGO_PCG_THREADS, 1) k_pgo_pcg(PcgArgs a) {
  __shared__ double sr[PGO_PCG_NODES][6];
  __shared__ double sp[PGO_PCG_STAGE][6];
  const unsigned int G = gridDim.x;
  const int N = a.N;
  const int npb = a.npb;
  const long long n6 = 6LL * N;
  const int groups = (N + npb - 1) / npb;
  const int ln = threadIdx.x / 6, row = threadIdx.x % 6;
  double tot[2];
  grid_total<2>(a.bpart, a.nbp, tot);
  const double bnorm = sqrt(tot[0]);
  if (bnorm == 0.0 || a.maxiter <= 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.st->pcg_iters = 0;
      a.st->pcg_rel = bnorm == 0.0 ? 0.0 : 1.0;
      a.st->pcg_done = 1;
    }
    return;
  }
  double* pA = a.p;
  double* pB = a.p + n6;
  // z = M r, rz
  double rz_part = 0.0;
  for (int gi = blockIdx.x; gi < groups; gi += G) {
    const int n = gi * npb + ln;
    const bool live = ln < npb && n < N;
    if (live) sr[ln][row] = a.r[6LL * n + row];
    __syncthreads();
    if (live) {
      const double* M = a.Minv + 36LL * n + 6 * row;
      double zz = 0.0;
      for (int k = 0; k < 6; ++k) zz += __ldg(M + k) * sr[ln][k];
      a.z[6LL * n + row] = zz;
      pA[6LL * n + row] = 0.0;
      rz_part += zz * sr[ln][row];
    }
    __syncthreads();
  }
  {
    double v[1] = {rz_part};
    block_sum_all<1>(v);
    if (threadIdx.x == 0) a.part[4LL * blockIdx.x] = v[0];
  }
  if (!grid_barrier(a.bar, G)) return;
  double rz;
  {
    double v[1] = {0.0};
    for (int i = threadIdx.x; i < (int)G; i += blockDim.x) v[0] += __ldcg(a.part + 4LL * i);
    block_sum_all<1>(v);
    rz = v[0];
  }
  double beta = 0.0;
  double rel = 1.0;
  int it = 0;
  double* pold = pA;
  double* pcur = pB;
  while (it < a.maxiter) {
    // phase A: p = z + beta p_old; q = (H + D) p; p . q
    double pq_part = 0.0;
    for (int gi = blockIdx.x; gi < groups; gi += G) {
      const int n0 = gi * npb;
      const int n = n0 + ln;
      const bool live = ln < npb && n < N;
      const bool free_n = live && !(a.fixed && a.fixed[n]);
      double pi[6];
      double pi_a = 0.0;
      if (live) {
#pragma unroll
        for (int k = 0; k < 6; ++k) pi[k] = __ldcg(a.z + 6LL * n + k) + beta * __ldcg(pold + 6LL * n + k);
        pi_a = __ldcg(a.z + 6LL * n + row) + beta * __ldcg(pold + 6LL * n + row);
      }
      double qa = 0.0;
      const int nend = min(N, n0 + npb);
      const int s_lo = __ldg(a.rowptr + n0), s_hi = __ldg(a.rowptr + nend);
      const int my_lo = live ? __ldg(a.rowptr + n) : 0, my_hi = live ? __ldg(a.rowptr + n + 1) : 0;
      for (int c0 = s_lo; c0 < s_hi; c0 += PGO_PCG_STAGE) {
        const int c1 = min(s_hi, c0 + PGO_PCG_STAGE);
        __syncthreads();
        for (int e = threadIdx.x; e < (c1 - c0) * 6; e += blockDim.x) {
          const int sl = e / 6, k = e % 6;
          const int other = __ldg(&a.inc2[c0 + sl].y);
          sp[sl][k] = __ldcg(a.z + 6LL * other + k) + beta * __ldcg(pold + 6LL * other + k);
        }
        __syncthreads();
        if (free_n) {
          const int lo = max(my_lo, c0), hi = min(my_hi, c1);
          for (int sl = lo; sl < hi; ++sl) {
            const int e = __ldg(&a.inc2[sl].x);
            const double* Br = a.B + 36LL * e + 6 * row;
            double acc = 0.0;
#pragma unroll
            for (int k = 0; k < 6; ++k) acc += __ldg(Br + k) * (pi[k] - sp[sl - c0][k]);
            qa += acc;
          }
        }
      }
      if (live) {
        const long long o = 6LL * n + row;
        pcur[o] = pi_a;
        if (free_n) qa += __ldg(a.D + o) * pi_a;
        else qa = 0.0;
        a.q[o] = qa;
        pq_part += pi_a * qa;
      }
    }
    {
      double v[1] = {pq_part};
      block_sum_all<1>(v);
      if (threadIdx.x == 0) a.part[4LL * blockIdx.x + 1] = v[0];
    }
    if (!grid_barrier(a.bar, G)) return;
    double pq;
    {
      double v[1] = {0.0};
      for (int i = threadIdx.x; i < (int)G; i += blockDim.x) v[0] += __ldcg(a.part + 4LL * i + 1);
      block_sum_all<1>(v);
      pq = v[0];
    }
    if (!(pq > 0.0)) break;
    const double alpha = rz / pq;
    // phase B: x += alpha p, r -= alpha q, z = M r; r . r, r . z
    double rr_part = 0.0, rzp = 0.0;
    for (int gi = blockIdx.x; gi < groups; gi += G) {
      const int n = gi * npb + ln;
      const bool live = ln < npb && n < N;
      if (live) {
        const long long o = 6LL * n + row;
        a.x[o] += alpha * pcur[o];
        const double rn = a.r[o] - alpha * a.q[o];
        a.r[o] = rn;
        sr[ln][row] = rn;
        rr_part += rn * rn;
      }
      __syncthreads();
      if (live) {
        const double* M = a.Minv + 36LL * n + 6 * row;
        double zz = 0.0;
        for (int k = 0; k < 6; ++k) zz += __ldg(M + k) * sr[ln][k];
        a.z[6LL * n + row] = zz;
        rzp += zz * sr[ln][row];
      }
      __syncthreads();
    }
    ++it;
    {
      double v[2] = {rr_part, rzp};
      block_sum_all<2>(v);
      if (threadIdx.x == 0) {
        a.part[4LL * blockIdx.x + 2] = v[0];
        a.part[4LL * blockIdx.x + 3] = v[1];
      }
    }
    if (!grid_barrier(a.bar, G)) return;
    double rr, rz_new;
    {
      double v[2] = {0.0, 0.0};
      for (int i = threadIdx.x; i < (int)G; i += blockDim.x) {
        v[0] += __ldcg(a.part + 4LL * i + 2);
        v[1] += __ldcg(a.part + 4LL * i + 3);
      }
      block_sum_all<2>(v);
      rr = v[0];
      rz_new = v[1];
    }
    rel = sqrt(rr) / bnorm;
    if (sqrt(rr) <= a.tol * bnorm) break;
    beta = rz_new / rz;
    rz = rz_new;
    double* t = pold;
    pold = pcur;
    pcur = t;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.st->pcg_iters = it;
    a.st->pcg_rel = it == 0 ? 1.0 : rel;
    a.st->pcg_done = 1;
  }
}

// Shared memory of k_pgo_pcg_res for a block of `slots` incidence slots:
// their B blocks (36), neighbour directions (6) and neighbour indices.
__host__ __device__ constexpr size_t pgo_res_smem(int slots) { return (size_t)slots * (36 * 8 + 6 * 8 + 4); }

// The same iteration as k_pgo_pcg when every block holds exactly one group
// of npb nodes (gridDim.x = ceil(N / npb)): each thread keeps its entry of
// x, r, z, p, D and its row of M for the whole solve in registers, the
// block's B blocks and neighbour indices are staged in shared memory once,
// and per iteration only the neighbours' z and p_old cross global memory.
// Same arithmetic, in the same order, as k_pgo_pcg.
static __global__ void __launch_bounds__(PGO_PCG_THREADS, 1) k_pgo_pcg_res(PcgArgs a) {
  extern __shared__ __align__(16) unsigned char pgo_smem[];
  __shared__ double sr[PGO_PCG_NODES][6];
  const unsigned int G = gridDim.x;
  const int N = a.N;
  const int npb = a.npb;
  const long long n6 = 6LL * N;
  const int ln = threadIdx.x / 6, row = threadIdx.x % 6;
  const int n0 = blockIdx.x * npb;
  const int n = n0 + ln;
  const bool live = ln < npb && n < N;
  const bool free_n = live && !(a.fixed && a.fixed[n]);
  const long long o = 6LL * n + row;
  const int nend = min(N, n0 + npb);
  const int s_lo = __ldg(a.rowptr + n0), s_hi = __ldg(a.rowptr + nend);
  const int nsl = s_hi - s_lo;
  double* sB = reinterpret_cast<double*>(pgo_smem);  // [nsl][36]
  double* sp = sB + 36LL * nsl;                      // [nsl][6]
  int* sother = reinterpret_cast<int*>(sp + 6LL * nsl);
  for (int e = threadIdx.x; e < nsl * 36; e += blockDim.x) {
    const int sl = e / 36, k = e % 36;
    sB[e] = __ldg(a.B + 36LL * __ldg(&a.inc2[s_lo + sl].x) + k);
  }
  for (int sl = threadIdx.x; sl < nsl; sl += blockDim.x) sother[sl] = __ldg(&a.inc2[s_lo + sl].y);
  const int my_lo = live ? __ldg(a.rowptr + n) - s_lo : 0, my_hi = live ? __ldg(a.rowptr + n + 1) - s_lo : 0;
  double Mrow[6];
  double Da = 0.0, ra = 0.0, xa = 0.0, za = 0.0, pa = 0.0;
  if (live) {
#pragma unroll
    for (int k = 0; k < 6; ++k) Mrow[k] = __ldg(a.Minv + 36LL * n + 6 * row + k);
    Da = __ldg(a.D + o);
    ra = a.r[o];
    sr[ln][row] = ra;
  }
  double tot[2];
  grid_total<2>(a.bpart, a.nbp, tot);  // ends with a block barrier: sr and the stages are complete
  const double bnorm = sqrt(tot[0]);
  if (bnorm == 0.0 || a.maxiter <= 0) {
    if (live) a.x[o] = 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.st->pcg_iters = 0;
      a.st->pcg_rel = bnorm == 0.0 ? 0.0 : 1.0;
      a.st->pcg_done = 1;
    }
    return;
  }
  double* pold = a.p;
  double* pcur = a.p + n6;
  double rz_part = 0.0;
  if (live) {
    double zz = 0.0;
#pragma unroll
    for (int k = 0; k < 6; ++k) zz += Mrow[k] * sr[ln][k];
    za = zz;
    a.z[o] = za;
    pold[o] = 0.0;
    rz_part = za * ra;
  }
  {
    double v[1] = {rz_part};
    block_sum_all<1>(v);
    if (threadIdx.x == 0) a.part[4LL * blockIdx.x] = v[0];
  }
  if (!grid_barrier(a.bar, G)) return;
  double rz;
  {
    double v[1] = {0.0};
    for (int i = threadIdx.x; i < (int)G; i += blockDim.x) v[0] += __ldcg(a.part + 4LL * i);
    block_sum_all<1>(v);
    rz = v[0];
  }
  double beta = 0.0;
  double rel = 1.0;
  int it = 0;
  while (it < a.maxiter) {
    // phase A: p = z + beta p_old; q = (H + D) p; p . q
    pa = za + beta * pa;
    if (live) {
      sr[ln][row] = pa;
      pcur[o] = pa;
    }
    for (int e = threadIdx.x; e < nsl * 6; e += blockDim.x) {
      const int sl = e / 6, k = e % 6;
      const long long g = 6LL * sother[sl] + k;
      sp[e] = __ldcg(a.z + g) + beta * __ldcg(pold + g);
    }
    __syncthreads();
    double qa = 0.0;
    if (free_n) {
      double pi[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) pi[k] = sr[ln][k];
      for (int sl = my_lo; sl < my_hi; ++sl) {
        const double* Br = sB + 36LL * sl + 6 * row;
        const double* po = sp + 6LL * sl;
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k) acc += Br[k] * (pi[k] - po[k]);
        qa += acc;
      }
      qa += Da * pa;
    }
    double pq_part = live ? pa * qa : 0.0;
    {
      double v[1] = {pq_part};
      block_sum_all<1>(v);
      if (threadIdx.x == 0) a.part[4LL * blockIdx.x + 1] = v[0];
    }
    if (!grid_barrier(a.bar, G)) return;
    double pq;
    {
      double v[1] = {0.0};
      for (int i = threadIdx.x; i < (int)G; i += blockDim.x) v[0] += __ldcg(a.part + 4LL * i + 1);
      block_sum_all<1>(v);
      pq = v[0];
    }
    if (!(pq > 0.0)) break;
    const double alpha = rz / pq;
    // phase B: x += alpha p, r -= alpha q, z = M r; r . r, r . z
    double rr_part = 0.0, rzp = 0.0;
    if (live) {
      xa += alpha * pa;
      ra = ra - alpha * qa;
      sr[ln][row] = ra;
      rr_part = ra * ra;
    }
    __syncthreads();
    if (live) {
      double zz = 0.0;
#pragma unroll
      for (int k = 0; k < 6; ++k) zz += Mrow[k] * sr[ln][k];
      za = zz;
      a.z[o] = za;
      rzp = za * ra;
    }
    ++it;
    {
      double v[2] = {rr_part, rzp};
      block_sum_all<2>(v);
      if (threadIdx.x == 0) {
        a.part[4LL * blockIdx.x + 2] = v[0];
        a.part[4LL * blockIdx.x + 3] = v[1];
      }
    }
    if (!grid_barrier(a.bar, G)) return;
    double rr, rz_new;
    {
      double v[2] = {0.0, 0.0};
      for (int i = threadIdx.x; i < (int)G; i += blockDim.x) {
        v[0] += __ldcg(a.part + 4LL * i + 2);
        v[1] += __ldcg(a.part + 4LL * i + 3);
      }
      block_sum_all<2>(v);
      rr = v[0];
      rz_new = v[1];
    }
    rel = sqrt(rr) / bnorm;
    if (sqrt(rr) <= a.tol * bnorm) break;
    beta = rz_new / rz;
    rz = rz_new;
    double* t = pold;
    pold = pcur;
    pcur = t;
  }
  if (live) a.x[o] = xa;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.st->pcg_iters = it;
    a.st->pcg_rel = it == 0 ? 1.0 : rel;
    a.st->pcg_done = 1;
  }
}

// y[6 pos[i] + a] = x[6 i + a] (to the factored order), or back (inverse).
static __global__ void k_pgo_permute(int N, const int32_t* __restrict__ pos, int inverse,
                                     const double* __restrict__ x, double* __restrict__ y) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 6LL * N) return;
  const int i = (int)(t / 6), a = (int)(t % 6);
  const long long o = 6LL * pos[i] + a;
  if (inverse) y[t] = x[o];
  else y[o] = x[t];
}

// ---------------------------------------------------------------------------
// Trial, cost and the LM decision
// ---------------------------------------------------------------------------

// Per node: zeta_i' = Exp(delta_i) zeta_i into the other pose buffer (a
// fixed node copies its pose), and the block partial of g . delta.
static __global__ void __launch_bounds__(PGO_NODE_THREADS)
k_pgo_trial(int N, const double* __restrict__ x, const double* __restrict__ g, const uint8_t* __restrict__ fixed,
            double* __restrict__ poses_buf, const DevState* st, double* __restrict__ part) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  double gd = 0.0;
  if (n < N) {
    const int cur = st->cur;
    const double* src = poses_buf + (long long)cur * 8 * N + 8LL * n;
    double* dst = poses_buf + (long long)(1 - cur) * 8 * N + 8LL * n;
    const Pose P = load_pose(src);
    double d[6];
    for (int k = 0; k < 6; ++k) {
      d[k] = x[6LL * n + k];
      gd += g[6LL * n + k] * d[k];
    }
    store_pose(dst, (fixed && fixed[n]) ? P : retract(P, d));
  }
  double v[1] = {gd};
  block_sum_store<1>(v, part + blockIdx.x);
}

// Per edge: 1/2 r^T Omega r at the poses of buffer (cur + which) % 2 and,
// when x is given, 1/2 u^T B u with u = x_j - x_i (the model's quadratic
// term); block partials [block][2].
static __global__ void __launch_bounds__(PGO_EDGE_THREADS)
k_pgo_edge_cost(int E, const int32_t* __restrict__ ei, const int32_t* __restrict__ ej,
                const double* __restrict__ meas, const double* __restrict__ info,
                const double* __restrict__ poses_buf, int N, const DevState* st, int which,
                const double* __restrict__ x, const double* __restrict__ B, double* __restrict__ part) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  double c = 0.0, quad = 0.0;
  if (e < E) {
    const double* poses = poses_buf + (long long)((st->cur + which) & 1) * 8 * N;
    const int i = ei[e], j = ej[e];
    const Pose Pi = load_pose(poses + 8LL * i);
    const Pose Pj = load_pose(poses + 8LL * j);
    const Pose Pm = load_pose(meas + 8LL * e);
    double qE[4], tE[3], r[6], Om[36];
    edge_error(Pi, Pj, Pm, qE, tE);
    se3_log(qE, tE, r);
    load_info(info + 21LL * e, Om);
    for (int a = 0; a < 6; ++a) {
      double t = 0.0;
      for (int b = 0; b < 6; ++b) t += Om[6 * a + b] * r[b];
      c += r[a] * t;
    }
    c *= 0.5;
    if (x) {
      double u[6];
      for (int k = 0; k < 6; ++k) u[k] = x[6LL * j + k] - x[6LL * i + k];
      const double* Be = B + 36LL * e;
      for (int a = 0; a < 6; ++a) {
        double t = 0.0;
        for (int b = 0; b < 6; ++b) t += Be[6 * a + b] * u[b];
        quad += u[a] * t;
      }
    }
  }
  double v[2] = {c, quad};
  block_sum_store<2>(v, part + 2LL * blockIdx.x);
}

// F at the current poses from k_pgo_edge_cost's partials (one block).
static __global__ void k_pgo_cost_set(int nb, const double* __restrict__ part, DevState* st) {
  const double F = block_sum_array(part, nb, 2);
  if (threadIdx.x == 0) {
    st->F = F;
    st->need_cost = 0;
  }
}

// Gain ratio, accept / reject and the damping update (one block), by the
// bundle-adjustment loop's rule: model = -g . delta - 1/2 delta^T H delta.
static __global__ void k_pgo_control(int nbe, const double* __restrict__ epart, int nbn,
                                     const double* __restrict__ gpart, int nbd, const double* __restrict__ dpart,
                                     double up, double down, double rho_good, double rho_bad, double lam_min,
                                     double lam_max, DevState* st, ba_iter_stats* __restrict__ stats, int cap) {
  const double Ft = block_sum_array(epart, nbe, 2);
  const double quad = block_sum_array(epart + 1, nbe, 2);
  const double lin = block_sum_array(gpart, nbn, 1);
  const double nbad = block_sum_array(dpart + 1, nbd, 2);
  if (threadIdx.x != 0) return;
  st->fallbacks = (int)nbad;
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
  }
  st->lam = nl;
  st->trials = t + 1;
}

// Block row i of H + D (6 rows, at block position pi = pos[i] of the
// factored order, or i without pos) into the band tiles of the banded
// Cholesky (tile size BAND_TB, half-bandwidth bwt tiles), lower triangle
// only: H_ii + D_i on the diagonal block, then -B_e at block (pi, po) for
// each incident edge whose other node comes earlier (po < pi), parallel
// edges summed in CSR order (one thread per block entry).  The rows and
// columns of a fixed node stay zero and its diagonal is 1.  The tiles are
// zeroed before.
static __global__ void __launch_bounds__(64)
k_pgo_band(int N, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ inc,
           const int32_t* __restrict__ ei, const int32_t* __restrict__ ej, const double* __restrict__ B,
           const double* __restrict__ Hd, const double* __restrict__ D, const int32_t* __restrict__ pos,
           const uint8_t* __restrict__ fixed, int bwt, double* __restrict__ T) {
  const int i = blockIdx.x, t = threadIdx.x;
  if (t >= 36) return;
  const int a = t / 6, b = t % 6;
  const int pi = pos ? pos[i] : i;
  const int R = 6 * pi + a;
  const bool fi = fixed && fixed[i];
  auto at = [&](int C) -> double& {
    const int I = R / BAND_TB, J = C / BAND_TB;
    return T[((long long)J * (bwt + 1) + (I - J)) * (BAND_TB * BAND_TB) + (R % BAND_TB) * BAND_TB + C % BAND_TB];
  };
  if (b <= a) at(6 * pi + b) = fi ? (a == b ? 1.0 : 0.0)
                                   : Hd[21LL * i + sym6(b, a)] + (a == b ? D[6LL * i + a] : 0.0);
  if (fi) return;
  const int end = rowptr[i + 1];
  for (int s = rowptr[i]; s < end; ++s) {
    const int code = inc[s];
    const int e = code >> 1;
    const int other = (code & 1) ? ei[e] : ej[e];
    const int po = pos ? pos[other] : other;
    if (po < pi && !(fixed && fixed[other])) at(6 * po + b) -= B[36LL * e + 6 * a + b];
  }
}

}  // namespace ba
