"""Pose-graph optimisation (PGO), the paper's second problem (Sec. IV-D,
"Generalization to Other Optimization Problems"): plain FP64 numpy, slow and
direct.  TEST INFRASTRUCTURE ONLY: the library never imports it.

Problem (Eq. 3): poses zeta_i in SE(3), edges (i, j) with a measured
relative pose T_ij and a 6x6 information matrix Omega_ij; minimise

    F(Z) = 1/2 sum_(i,j) r_ij^T Omega_ij r_ij,
    r_ij = Log(zeta_i^{-1} zeta_j T_ij^{-1})          (Eq. 4)

with the same LM loop as bundle adjustment (Alg. 1).  Readings (the paper
leaves them to PyPose's LieTensor):
  - tangent vectors are xi = (rho, phi): translation part first, rotation
    part second; hat(xi) = [[phi^, rho], [0, 0]] (4 x 4);
  - an update is the left retraction zeta <- Exp(delta) zeta;
  - the cost carries the factor 1/2 of the bundle-adjustment cost, so its
    gradient is J^T Omega r;
  - a pose marked fixed never moves (the gauge: PGO's cost is invariant
    under zeta_i <- G zeta_i for every i).

Derivatives: with E = zeta_i^{-1} zeta_j T_ij^{-1}, perturbing zeta_j by
Exp(delta) gives E' = Exp(Ad(zeta_i^{-1}) delta) E, perturbing zeta_i gives
E' = Exp(-Ad(zeta_i^{-1}) delta) E, and Log(Exp(a) E) = r + J_l(r)^{-1} a +
O(|a|^2).  So dr/d(delta_j) = A, dr/d(delta_i) = -A with
A = J_l(r)^{-1} Ad(zeta_i^{-1}), and every edge adds B = A^T Omega A to both
diagonal blocks of H = J^T Omega J and -B to the two off-diagonal ones.

Here every map is taken from its definition: Exp is the matrix exponential
of hat(xi), Ad and ad are read off conjugation and the Lie bracket, and the
left Jacobian is the series sum_n ad^n / (n+1)!, evaluated exactly as a
block of the exponential of [[ad, I], [0, 0]].  Log is the only closed form:
the rotation vector (scipy), then rho = J_l^{SO(3)}(phi)^{-1} t.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sl
from scipy.spatial.transform import Rotation

from .ba_oracle import LMOptions, cholesky_solve, damp_diag, left_jacobian, pcg, skew


# --------------------------------------------------------------------------
# SE(3)
# --------------------------------------------------------------------------

def hat6(xi):
    """The 4 x 4 matrix of the tangent vector xi = (rho, phi)."""
    xi = np.asarray(xi, dtype=np.float64)
    X = np.zeros((4, 4))
    X[:3, :3] = skew(xi[3:6])
    X[:3, 3] = xi[0:3]
    return X


def vee6(X):
    """Inverse of hat6 (reads the translation column and the skew part)."""
    return np.array([X[0, 3], X[1, 3], X[2, 3], X[2, 1], X[0, 2], X[1, 0]])


def se3_exp(xi):
    """Exp(xi): the matrix exponential of hat(xi) (definition)."""
    return sl.expm(hat6(xi))


def se3_log(T):
    """Log(T) = (rho, phi): phi the rotation vector of R (|phi| <= pi), rho =
    J_l(phi)^{-1} t (the translation of Exp(rho, phi) is J_l(phi) rho)."""
    T = np.asarray(T, dtype=np.float64)
    phi = Rotation.from_matrix(T[:3, :3]).as_rotvec()
    rho = np.linalg.solve(left_jacobian(phi), T[:3, 3])
    return np.concatenate([rho, phi])


def se3_inv(T):
    Ti = np.eye(4)
    R = T[:3, :3]
    Ti[:3, :3] = R.T
    Ti[:3, 3] = -R.T @ T[:3, 3]
    return Ti


def adjoint(T):
    """Ad(T), 6 x 6: column k is vee(T hat(e_k) T^{-1}), so that
    T Exp(xi) T^{-1} = Exp(Ad(T) xi)."""
    Ti = se3_inv(T)
    A = np.zeros((6, 6))
    for k in range(6):
        e = np.zeros(6)
        e[k] = 1.0
        A[:, k] = vee6(T @ hat6(e) @ Ti)
    return A


def ad(xi):
    """ad(xi), 6 x 6: column k is vee([hat(xi), hat(e_k)]) (the Lie bracket)."""
    X = hat6(xi)
    A = np.zeros((6, 6))
    for k in range(6):
        e = np.zeros(6)
        e[k] = 1.0
        E = hat6(e)
        A[:, k] = vee6(X @ E - E @ X)
    return A


def left_jacobian_se3(xi):
    """J_l(xi) = sum_n ad(xi)^n / (n+1)! = int_0^1 exp(s ad(xi)) ds: the
    upper-right block of exp([[ad, I], [0, 0]])."""
    M = np.zeros((12, 12))
    M[:6, :6] = ad(xi)
    M[:6, 6:] = np.eye(6)
    return sl.expm(M)[:6, 6:]


# --------------------------------------------------------------------------
# Pose formats
# --------------------------------------------------------------------------

def pose_matrix(p7):
    """(tx, ty, tz, qx, qy, qz, qw) -> 4 x 4 (the quaternion need not be
    normalised)."""
    p7 = np.asarray(p7, dtype=np.float64)
    T = np.eye(4)
    T[:3, :3] = Rotation.from_quat(p7[3:7]).as_matrix()
    T[:3, 3] = p7[0:3]
    return T


def pose_vector(T):
    """4 x 4 -> (t, q) with a unit quaternion, qw >= 0."""
    q = Rotation.from_matrix(T[:3, :3]).as_quat()
    if q[3] < 0:
        q = -q
    return np.concatenate([T[:3, 3], q])


def poses_to_matrices(P7):
    return np.stack([pose_matrix(p) for p in np.asarray(P7)])


def matrices_to_poses(Ts):
    return np.stack([pose_vector(T) for T in Ts])


def info_matrix(u21):
    """The 6 x 6 symmetric matrix of its upper triangle, row by row
    ((0,0), (0,1), ..., (0,5), (1,1), ..., (5,5))."""
    M = np.zeros((6, 6))
    k = 0
    for a in range(6):
        for b in range(a, 6):
            M[a, b] = M[b, a] = u21[k]
            k += 1
    return M


def info_upper(M):
    return np.array([M[a, b] for a in range(6) for b in range(a, 6)])


def graph_inputs(graph):
    """A scenegen PoseGraph's arrays as matrices: the initial estimate
    Exp(drift_i) zeta_i, the measurements T_ij = Exp(noise_e) zeta_i^{-1}
    zeta_j and the 6 x 6 information matrices.  Returns (Ts_init [N,4,4],
    Tms [E,4,4], infos [E,6,6], Ts_gt [N,4,4])."""
    Tg = poses_to_matrices(graph.poses_gt)
    Ts = np.stack([se3_exp(d) @ T for d, T in zip(graph.drift, Tg)])
    Tms = np.stack([se3_exp(n) @ se3_inv(Tg[i]) @ Tg[j] for n, i, j in zip(graph.noise, graph.ei, graph.ej)])
    infos = np.stack([info_matrix(u) for u in graph.info])
    return Ts, Tms, infos, Tg


# --------------------------------------------------------------------------
# Residuals, Jacobians, normal equations
# --------------------------------------------------------------------------

def edge_error(Ti, Tj, Tm):
    """E = zeta_i^{-1} zeta_j T_ij^{-1}."""
    return se3_inv(Ti) @ Tj @ se3_inv(Tm)


def residual(Ti, Tj, Tm):
    """r_ij = Log(zeta_i^{-1} zeta_j T_ij^{-1}) (Eq. 4)."""
    return se3_log(edge_error(Ti, Tj, Tm))


def edge_jacobian(Ti, Tj, Tm):
    """A = dr/d(delta_j) = J_l(r)^{-1} Ad(zeta_i^{-1}); dr/d(delta_i) = -A."""
    r = residual(Ti, Tj, Tm)
    return np.linalg.solve(left_jacobian_se3(r), adjoint(se3_inv(Ti)))


def residuals(Ts, ei, ej, Tms):
    return np.stack([residual(Ts[i], Ts[j], Tm) for i, j, Tm in zip(ei, ej, Tms)])


def cost(Ts, ei, ej, Tms, infos):
    """F = 1/2 sum_e r_e^T Omega_e r_e (numpy's pairwise sum of the terms)."""
    r = residuals(Ts, ei, ej, Tms)
    terms = np.einsum("ea,eab,eb->e", r, infos, r)
    return 0.5 * float(np.sum(terms))


def assemble(Ts, ei, ej, Tms, infos):
    """Per-edge r [E,6], A [E,6,6], B = A^T Omega A, q = A^T Omega r; per
    node the diagonal blocks H_ii = sum_{e at i} B_e [N,6,6] and the
    gradient g = J^T Omega r [N,6] (g_i -= q_e, g_j += q_e)."""
    N = len(Ts)
    E = len(ei)
    r = np.zeros((E, 6))
    A = np.zeros((E, 6, 6))
    for e in range(E):
        Ti, Tj, Tm = Ts[ei[e]], Ts[ej[e]], Tms[e]
        r[e] = residual(Ti, Tj, Tm)
        A[e] = np.linalg.solve(left_jacobian_se3(r[e]), adjoint(se3_inv(Ti)))
    B = np.einsum("eka,ekl,elb->eab", A, infos, A)
    q = np.einsum("eka,ekl,el->ea", A, infos, r)
    Hd = np.zeros((N, 6, 6))
    g = np.zeros((N, 6))
    for e in range(E):
        Hd[ei[e]] += B[e]
        Hd[ej[e]] += B[e]
        g[ei[e]] -= q[e]
        g[ej[e]] += q[e]
    return dict(r=r, A=A, B=B, q=q, Hd=Hd, g=g, ei=np.asarray(ei), ej=np.asarray(ej), N=N)


def dense_jacobian(blk):
    """J [6E, 6N] from the edge blocks (-A at node i, A at node j)."""
    E = len(blk["ei"])
    J = np.zeros((6 * E, 6 * blk["N"]))
    for e in range(E):
        i, j = blk["ei"][e], blk["ej"][e]
        J[6 * e:6 * e + 6, 6 * i:6 * i + 6] -= blk["A"][e]
        J[6 * e:6 * e + 6, 6 * j:6 * j + 6] += blk["A"][e]
    return J


def hessian_dense(blk):
    """H = J^T Omega J assembled block by block (6N x 6N)."""
    N = blk["N"]
    H = np.zeros((6 * N, 6 * N))
    for e, (i, j) in enumerate(zip(blk["ei"], blk["ej"])):
        B = blk["B"][e]
        H[6 * i:6 * i + 6, 6 * i:6 * i + 6] += B
        H[6 * j:6 * j + 6, 6 * j:6 * j + 6] += B
        H[6 * i:6 * i + 6, 6 * j:6 * j + 6] -= B
        H[6 * j:6 * j + 6, 6 * i:6 * i + 6] -= B
    return H


def matvec(blk, x):
    """(H x)_i = sum over the edges e at node i of B_e (x_i - x_other(e))."""
    y = np.zeros_like(x)
    for e, (i, j) in enumerate(zip(blk["ei"], blk["ej"])):
        d = blk["B"][e] @ (x[i] - x[j])
        y[i] += d
        y[j] -= d
    return y


def damping(blk, lam, opts):
    """lambda clamp(diag H_ii) per node [N, 6] (Alg. 1's damping term)."""
    diag = np.einsum("naa->na", blk["Hd"])
    return damp_diag(diag, lam, opts.diag_min, opts.diag_max)


def solve_damped(blk, lam, opts, fixed=None):
    """Solve (H + D) delta = -g over the free nodes (fixed nodes: delta = 0)
    with block-Jacobi PCG (6 x 6 blocks of H + D) or a dense Cholesky.
    Returns (delta [N,6], iterations, |r|/|b|)."""
    N = blk["N"]
    free = np.ones(N, bool) if fixed is None else ~np.asarray(fixed, bool)
    D = damping(blk, lam, opts)
    b = -blk["g"] * free[:, None]
    if opts.solver == "cholesky":
        H = hessian_dense(blk) + np.diag(D.reshape(-1))
        keep = np.repeat(free, 6)
        x = np.zeros(6 * N)
        x[keep] = cholesky_solve(H[np.ix_(keep, keep)], b.reshape(-1)[keep])
        return x.reshape(N, 6), 0, 0.0
    Hs = blk["Hd"].copy()
    idx = np.arange(6)
    Hs[:, idx, idx] += D
    Minv = np.linalg.inv(Hs) * free[:, None, None]

    def mv(x):
        x = x * free[:, None]
        return (matvec(blk, x) + D * x) * free[:, None]

    def pre(r):
        return np.einsum("nab,nb->na", Minv, r)

    x, its, rel = pcg(mv, pre, b, opts.pcg_tol, opts.pcg_maxiter)
    return x, its, rel


def retract(Ts, delta):
    """zeta_i <- Exp(delta_i) zeta_i."""
    return np.stack([se3_exp(d) @ T for d, T in zip(delta, Ts)])


def model_reduction(blk, delta):
    """Delta L = -g^T delta - 1/2 delta^T H delta, the last term as
    1/2 sum_e (delta_j - delta_i)^T B_e (delta_j - delta_i)."""
    u = delta[blk["ej"]] - delta[blk["ei"]]
    quad = float(np.sum(np.einsum("ea,eab,eb->e", u, blk["B"], u)))
    return -float(np.sum(blk["g"] * delta)) - 0.5 * quad


def lm(Ts0, ei, ej, Tms, infos, iters, opts=None, fixed=None):
    """The LM loop of Alg. 1 on the pose graph, with the bundle-adjustment
    loop's acceptance and damping rules (accept when F' is finite, Delta L >
    0 and F' < F; lambda /= up when rho > rho_good, lambda /= down when
    rejected or rho < rho_bad).  Returns (poses [N,4,4], trace)."""
    opts = opts or LMOptions()
    Ts = np.array(Ts0, dtype=np.float64, copy=True)
    lam = opts.lambda0
    F = cost(Ts, ei, ej, Tms, infos)
    blk = None
    trace = []
    for _ in range(iters):
        if blk is None:
            blk = assemble(Ts, ei, ej, Tms, infos)
        delta, its, rel = solve_damped(blk, lam, opts, fixed)
        Tt = retract(Ts, delta)
        Ft = cost(Tt, ei, ej, Tms, infos)
        dL = model_reduction(blk, delta)
        rho = (F - Ft) / dL if dL != 0.0 else float("nan")
        accept = bool(np.isfinite(Ft) and dL > 0.0 and Ft < F)
        trace.append(dict(cost=F, cost_trial=Ft, model=dL, rho=rho, lam=lam, accepted=accept, pcg_iters=its,
                          pcg_rel_res=rel))
        if accept:
            Ts, F = Tt, Ft
            blk = None
            if rho > opts.rho_good:
                lam = max(lam / opts.up, opts.lambda_min)
            elif rho < opts.rho_bad:
                lam = min(lam / opts.down, opts.lambda_max)
        else:
            lam = min(lam / opts.down, opts.lambda_max)
    return Ts, trace
