"""Plain FP64 reference for the LM bundle-adjustment hot path.

TEST INFRASTRUCTURE ONLY -- see the package docstring.  Everything here is
float64 numpy, written for a reader who checks it against the paper by eye:
vectorised over observations, no blocking, no fusion; per-block sums are
taken in observation-index order (``np.bincount``).

What it computes, by the paper's section:

* Eq. 1 (Sec. III-A): the non-linear least-squares objective, a sum over the
  observed (camera, point) pairs only.  Read here as F = 1/2 sum rho(|r_k|^2)
  with r_k = pi(theta_c(k), X_p(k)) - x_k, rho the identity or Huber's loss.
* Sec. III-C: every residual touches exactly one camera block and one point
  block, so J is stored as per-observation 2x9 / 2x3 blocks.
* Alg. 1 and Eq. 2 (Sec. III-B): A = J^T J, A + lambda diag(A), solve
  A dtheta = -J^T R, update lambda, theta += dtheta.
* Sec. IV-B: the "symbolic phase" (which blocks multiply into which) depends
  only on the index pattern; here it is the stable sort of the observations by
  camera and by point (``csr_build``).
* Sec. IV-B (diagonal clamping): diag(A) is clamped into [diag_min, diag_max]
  before it is scaled by lambda.
* Sec. IV-C: the linear solve, either a direct Cholesky factorisation or a
  preconditioned conjugate gradient; the minimum code example fixes
  PCG(tol=1e-4, maxiter=250) and TrustRegion(up=2.0, down=0.5**4).

Not in the paper, and read as follows:

* camera model: the 9-parameter BAL camera of the paper's benchmark data
  (angle-axis omega, translation t, focal f, radial k1, k2); X_cam = R(omega)X+t,
  p = -X_cam[:2]/X_cam[2] (the sign of the paper's ``project``), distortion
  1 + k1|p|^2 + k2|p|^4, pixel = f * distortion * p.  All nine parameters and
  the point update additively.
* the reduced camera system (Schur complement of the point blocks) solved by
  PCG with a 9x9 block-Jacobi preconditioner and an implicit S x product;
* Huber's loss on the residual norm, used as IRLS weights w = rho'(s);
* the trust-region rule (``LMOptions``) and the gain ratio's model reduction
  Delta L = -g^T Delta - 1/2 sum_k w_k |J_k Delta|^2.
"""
from __future__ import annotations

import dataclasses

import numpy as np

__all__ = [
    "skew", "rodrigues", "left_jacobian", "project", "residuals",
    "huber", "cost", "linearize", "csr_build", "segment_sum", "assemble",
    "dense_jacobian", "damp_diag", "point_damped_inverse", "schur_explicit",
    "schur_matvec", "block_jacobi", "pcg", "cholesky_solve", "back_substitute",
    "model_reduction", "solve_damped", "LMOptions", "lm", "dense_lm_delta",
    "gauge_transform", "pixels_from_scene", "gauge_mask", "adjoint_dense",
    "adjoint_schur",
]


# --------------------------------------------------------------------------
# SO(3) and the camera model
# --------------------------------------------------------------------------

def skew(v):
    """[v]_x such that [v]_x u = v x u; v has shape [..., 3]."""
    v = np.asarray(v, dtype=np.float64)
    z = np.zeros(v.shape[:-1])
    return np.stack([
        np.stack([z, -v[..., 2], v[..., 1]], -1),
        np.stack([v[..., 2], z, -v[..., 0]], -1),
        np.stack([-v[..., 1], v[..., 0], z], -1),
    ], -2)


def _so3_coeffs(omega):
    """a = sin(th)/th, b = (1-cos(th))/th^2, c = (th - sin(th))/th^3.

    b is taken from the half-angle form 2 sin^2(th/2)/th^2, which has no
    cancellation; a and b switch to their Taylor series below th = 1e-4 and c
    below th = 0.1 (where th - sin(th) cancels), each truncated after a term
    smaller than 1e-16 relative.
    """
    th2 = np.sum(np.asarray(omega, dtype=np.float64) ** 2, axis=-1)
    th = np.sqrt(th2)
    with np.errstate(divide="ignore", invalid="ignore"):
        a = np.where(th < 1e-4, 1.0 - th2 / 6.0, np.sin(th) / th)
        half = np.sin(0.5 * th)
        b = np.where(th < 1e-4, 0.5 - th2 / 24.0, 2.0 * half * half / th2)
        c = np.where(th < 0.1,
                     1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0
                     - th2 * th2 * th2 / 362880.0,
                     (th - np.sin(th)) / (th2 * th))
    return a, b, c


def rodrigues(omega):
    """R(omega) = I + a [w]_x + b [w]_x^2 (Rodrigues' formula)."""
    omega = np.asarray(omega, dtype=np.float64)
    a, b, _ = _so3_coeffs(omega)
    K = skew(omega)
    I = np.broadcast_to(np.eye(3), K.shape)
    return I + a[..., None, None] * K + b[..., None, None] * (K @ K)


def left_jacobian(omega):
    """J_l(omega) = I + b [w]_x + c [w]_x^2, so that
    R(omega + d) = (I + [J_l d]_x) R(omega) + O(|d|^2)."""
    omega = np.asarray(omega, dtype=np.float64)
    _, b, c = _so3_coeffs(omega)
    K = skew(omega)
    I = np.broadcast_to(np.eye(3), K.shape)
    return I + b[..., None, None] * K + c[..., None, None] * (K @ K)


def _camera_point(cams, points, cam_idx, pt_idx):
    cams = np.asarray(cams, dtype=np.float64)
    points = np.asarray(points, dtype=np.float64)
    cam = cams[cam_idx]
    R = rodrigues(cam[:, 0:3])
    X = points[pt_idx]
    RX = np.einsum("oij,oj->oi", R, X)
    Pc = RX + cam[:, 3:6]
    return cam, R, X, RX, Pc


def project(cams, points, cam_idx, pt_idx):
    """pi(theta_c, X) per observation, shape [O, 2] (the BAL camera)."""
    cam, _, _, _, Pc = _camera_point(cams, points, cam_idx, pt_idx)
    p = -Pc[:, 0:2] / Pc[:, 2:3]
    r2 = np.sum(p * p, axis=1)
    dist = 1.0 + cam[:, 7] * r2 + cam[:, 8] * r2 * r2
    return (cam[:, 6] * dist)[:, None] * p


def residuals(cams, points, cam_idx, pt_idx, pixels):
    """r_k = pi(theta_c(k), X_p(k)) - x_k (the residual of Eq. 1)."""
    return project(cams, points, cam_idx, pt_idx) - np.asarray(pixels, np.float64)


def huber(s, delta):
    """Loss rho(s) and IRLS weight w = rho'(s) of the squared norm s = |r|^2.

    delta <= 0: rho(s) = s, w = 1.  Otherwise Huber on |r|: rho(s) = s for
    s <= delta^2, else 2 delta sqrt(s) - delta^2, and w = min(1, delta/sqrt(s)).
    """
    s = np.asarray(s, dtype=np.float64)
    if delta is None or delta <= 0.0:
        return s.copy(), np.ones_like(s)
    inl = s <= delta * delta
    sq = np.sqrt(s)
    with np.errstate(divide="ignore", invalid="ignore"):
        rho = np.where(inl, s, 2.0 * delta * sq - delta * delta)
        w = np.where(inl, 1.0, delta / sq)
    return rho, w


def cost(cams, points, cam_idx, pt_idx, pixels, delta=0.0):
    """F(theta) = 1/2 sum_k rho(|r_k|^2) (numpy's pairwise sum)."""
    r = residuals(cams, points, cam_idx, pt_idx, pixels)
    rho, _ = huber(np.sum(r * r, axis=1), delta)
    return 0.5 * float(np.sum(rho))


def linearize(cams, points, cam_idx, pt_idx, pixels):
    """Residuals and analytic Jacobian blocks.

    Returns r [O,2], Jc [O,2,9] = d r / d(omega, t, f, k1, k2) and
    Jp [O,2,3] = d r / d X, by the chain rule through
      X_cam = R X + t,  p = -X_cam[:2]/X_cam[2],  d = 1 + k1|p|^2 + k2|p|^4,
      pi = f d p:
      d pi/d p     = f d I + f (2 k1 + 4 k2 |p|^2) p p^T
      d p/d X_cam  = -(1/X_cam[2]) [[1, 0, p_x], [0, 1, p_y]]
      d X_cam/d omega = -[R X]_x J_l(omega),  d X_cam/d t = I,
      d X_cam/d X  = R,
      d pi/d f = d p,  d pi/d k1 = f |p|^2 p,  d pi/d k2 = f |p|^4 p.
    """
    cam, R, X, RX, Pc = _camera_point(cams, points, cam_idx, pt_idx)
    O = Pc.shape[0]
    f = cam[:, 6]
    k1 = cam[:, 7]
    k2 = cam[:, 8]
    p = -Pc[:, 0:2] / Pc[:, 2:3]
    r2 = np.sum(p * p, axis=1)
    dist = 1.0 + k1 * r2 + k2 * r2 * r2
    r = (f * dist)[:, None] * p - np.asarray(pixels, np.float64)

    dpi_dp = (f * dist)[:, None, None] * np.eye(2)[None] + \
        (f * (2.0 * k1 + 4.0 * k2 * r2))[:, None, None] * np.einsum("oi,oj->oij", p, p)
    dp_dP = np.zeros((O, 2, 3))
    inv_z = -1.0 / Pc[:, 2]
    dp_dP[:, 0, 0] = inv_z
    dp_dP[:, 1, 1] = inv_z
    dp_dP[:, 0, 2] = inv_z * p[:, 0]
    dp_dP[:, 1, 2] = inv_z * p[:, 1]
    A = dpi_dp @ dp_dP                                    # d pi / d X_cam
    dP_dom = -skew(RX) @ left_jacobian(cam[:, 0:3])
    Jc = np.empty((O, 2, 9))
    Jc[:, :, 0:3] = A @ dP_dom
    Jc[:, :, 3:6] = A
    Jc[:, :, 6] = dist[:, None] * p
    Jc[:, :, 7] = (f * r2)[:, None] * p
    Jc[:, :, 8] = (f * r2 * r2)[:, None] * p
    Jp = A @ R
    return r, Jc, Jp


# --------------------------------------------------------------------------
# Symbolic phase: stable CSR of the observations by camera and by point
# --------------------------------------------------------------------------

def csr_build(keys, n_keys):
    """Stable sort of observation indices by key, plus the row pointer.

    perm lists the observations of key 0 in increasing index order, then key 1,
    ...; rowptr[i]:rowptr[i+1] is key i's range (a counting sort; numpy's
    stable argsort is that sort)."""
    keys = np.asarray(keys, dtype=np.int64)
    perm = np.argsort(keys, kind="stable").astype(np.int32)
    counts = np.bincount(keys, minlength=n_keys)
    rowptr = np.zeros(n_keys + 1, dtype=np.int32)
    rowptr[1:] = np.cumsum(counts)
    return perm, rowptr


def segment_sum(idx, vals, n):
    """out[i] = sum of vals[k] over k with idx[k] == i, in index order."""
    vals = np.asarray(vals, dtype=np.float64)
    flat = vals.reshape(vals.shape[0], -1)
    out = np.empty((n, flat.shape[1]))
    for c in range(flat.shape[1]):
        out[:, c] = np.bincount(idx, weights=flat[:, c], minlength=n)
    return out.reshape((n,) + vals.shape[1:])


# --------------------------------------------------------------------------
# Normal equations in blocks (Alg. 1, A = J^T J and -J^T R)
# --------------------------------------------------------------------------

def assemble(cams, points, cam_idx, pt_idx, pixels, delta=0.0):
    """Block normal equations with IRLS weights w_k = rho'(|r_k|^2):

    U_i = sum_{k in cam i} w Jc^T Jc,  V_j = sum_{k in pt j} w Jp^T Jp,
    W_k = w Jc_k^T Jp_k,  gc_i = sum w Jc^T r,  gp_j = sum w Jp^T r,
    F = 1/2 sum rho.
    """
    C = np.asarray(cams).shape[0]
    P = np.asarray(points).shape[0]
    r, Jc, Jp = linearize(cams, points, cam_idx, pt_idx, pixels)
    s = np.sum(r * r, axis=1)
    rho, w = huber(s, delta)
    U = segment_sum(cam_idx, w[:, None, None] * np.einsum("oai,oaj->oij", Jc, Jc), C)
    V = segment_sum(pt_idx, w[:, None, None] * np.einsum("oai,oaj->oij", Jp, Jp), P)
    W = w[:, None, None] * np.einsum("oai,oaj->oij", Jc, Jp)
    gc = segment_sum(cam_idx, w[:, None] * np.einsum("oai,oa->oi", Jc, r), C)
    gp = segment_sum(pt_idx, w[:, None] * np.einsum("oai,oa->oi", Jp, r), P)
    return dict(r=r, Jc=Jc, Jp=Jp, w=w, U=U, V=V, W=W, gc=gc, gp=gp,
                F=0.5 * float(np.sum(rho)))


def dense_jacobian(cams, points, cam_idx, pt_idx, pixels, delta=0.0):
    """The full weighted Jacobian sqrt(w) J, shape [2O, 9C + 3P], and sqrt(w) r.

    Column layout: camera i's 9 parameters at 9i, point j's 3 at 9C + 3j."""
    C = np.asarray(cams).shape[0]
    P = np.asarray(points).shape[0]
    r, Jc, Jp = linearize(cams, points, cam_idx, pt_idx, pixels)
    _, w = huber(np.sum(r * r, axis=1), delta)
    sw = np.sqrt(w)
    O = r.shape[0]
    J = np.zeros((2 * O, 9 * C + 3 * P))
    for k in range(O):
        c = int(cam_idx[k])
        j = int(pt_idx[k])
        J[2 * k:2 * k + 2, 9 * c:9 * c + 9] += sw[k] * Jc[k]
        J[2 * k:2 * k + 2, 9 * C + 3 * j:9 * C + 3 * j + 3] += sw[k] * Jp[k]
    return J, (sw[:, None] * r).reshape(-1)


def damp_diag(diag, lam, diag_min, diag_max):
    """lambda * clamp(diag, diag_min, diag_max): the term Alg. 1 adds to A."""
    return lam * np.clip(diag, diag_min, diag_max)


def point_damped_inverse(V, lam, diag_min, diag_max):
    """V*_j = V_j + lambda clamp(diag V_j); returns V*^{-1} [P,3,3]."""
    Vs = V.copy()
    idx = np.arange(3)
    Vs[:, idx, idx] += damp_diag(V[:, idx, idx], lam, diag_min, diag_max)
    return np.linalg.inv(Vs)


def _ustar(U, lam, diag_min, diag_max):
    Us = U.copy()
    idx = np.arange(9)
    Us[:, idx, idx] += damp_diag(U[:, idx, idx], lam, diag_min, diag_max)
    return Us


def schur_explicit(blk, cam_idx, pt_idx, lam, diag_min=1e-6, diag_max=1e32):
    """Dense reduced camera system S dc = b of the damped normal equations.

    [U* W; W^T V*] [dc; dp] = -[gc; gp]  gives
    S = U* - W V*^{-1} W^T,  b = -gc + W V*^{-1} gp,
    built pair by pair over the observations of each point (so repeated
    (camera, point) pairs are also exact)."""
    U, V, W, gc, gp = blk["U"], blk["V"], blk["W"], blk["gc"], blk["gp"]
    C = U.shape[0]
    P = V.shape[0]
    Us = _ustar(U, lam, diag_min, diag_max)
    Vinv = point_damped_inverse(V, lam, diag_min, diag_max)
    cam_idx = np.asarray(cam_idx, dtype=np.int64)
    pt_idx = np.asarray(pt_idx, dtype=np.int64)
    # every ordered pair (k, l) of observations of the same point
    perm, rowptr = csr_build(pt_idx, P)
    cnt = np.diff(rowptr).astype(np.int64)
    pos_pt = np.repeat(np.arange(P), cnt)              # point of each sorted slot
    n_of = cnt[pos_pt]
    a = np.repeat(np.arange(perm.shape[0]), n_of)      # slot of k, repeated
    first = np.repeat(np.cumsum(n_of) - n_of, n_of)
    bslot = rowptr[pos_pt[a]] + (np.arange(a.shape[0]) - first)
    k = perm[a].astype(np.int64)
    l = perm[bslot].astype(np.int64)
    j = pos_pt[a]
    blocks = W[k] @ Vinv[j] @ np.transpose(W[l], (0, 2, 1))
    S4 = segment_sum(cam_idx[k] * C + cam_idx[l], blocks, C * C).reshape(C, C, 9, 9)
    S = -S4.transpose(0, 2, 1, 3).reshape(9 * C, 9 * C)
    for i in range(C):
        S[9 * i:9 * i + 9, 9 * i:9 * i + 9] += Us[i]
    y = np.einsum("pij,pj->pi", Vinv, gp)
    b = (-gc + segment_sum(cam_idx, np.einsum("oij,oj->oi", W, y[pt_idx]), C)).reshape(-1)
    return S, b, Us, Vinv


def schur_matvec(x, Us, Vinv, W, cam_idx, pt_idx):
    """S x = U* x - W (V*^{-1} (W^T x)), never forming S.  x has shape [C, 9]."""
    C = Us.shape[0]
    P = Vinv.shape[0]
    z = segment_sum(pt_idx, np.einsum("oij,oi->oj", W, x[cam_idx]), P)
    y = np.einsum("pij,pj->pi", Vinv, z)
    return np.einsum("cij,cj->ci", Us, x) - \
        segment_sum(cam_idx, np.einsum("oij,oj->oi", W, y[pt_idx]), C)


def block_jacobi(Us, Vinv, W, cam_idx, pt_idx):
    """M_i = (U*_i - sum_{k in cam i} W_k V*^{-1}_{p(k)} W_k^T)^{-1}.

    The sum is the 9x9 diagonal block of W V*^{-1} W^T when no (camera, point)
    pair is observed twice."""
    C = Us.shape[0]
    WVW = W @ Vinv[pt_idx] @ np.transpose(W, (0, 2, 1))
    return np.linalg.inv(Us - segment_sum(cam_idx, WVW, C))


def pcg(matvec, precond, b, tol, maxiter):
    """Preconditioned conjugate gradient from x0 = 0 (Sec. IV-C).

    Stops after the first iteration whose residual satisfies
    |r| <= tol |b| (2-norms), or after maxiter iterations, or when the
    curvature p^T S p is not positive.  Returns (x, iterations, |r|/|b|)."""
    x = np.zeros_like(b)
    r = b.copy()
    bnorm = float(np.sqrt(np.sum(b * b)))
    if bnorm == 0.0 or maxiter <= 0:
        return x, 0, 0.0 if bnorm == 0.0 else 1.0
    z = precond(r)
    p = z.copy()
    rz = float(np.sum(r * z))
    it = 0
    while it < maxiter:
        q = matvec(p)
        pq = float(np.sum(p * q))
        if not pq > 0.0:
            break
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        if float(np.sqrt(np.sum(r * r))) <= tol * bnorm:
            break
        z = precond(r)
        rz_new = float(np.sum(r * z))
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
    return x, it, float(np.sqrt(np.sum(r * r))) / bnorm


def cholesky_solve(S, b):
    """Solve S x = b with a dense Cholesky factorisation S = L L^T."""
    import scipy.linalg as sl
    L = np.linalg.cholesky(S)
    y = sl.solve_triangular(L, b, lower=True)
    return sl.solve_triangular(L.T, y, lower=False)


def back_substitute(dc, blk, Vinv, cam_idx, pt_idx):
    """dp_j = V*_j^{-1} (-gp_j - sum_{k in pt j} W_k^T dc_c(k))."""
    P = Vinv.shape[0]
    z = segment_sum(pt_idx, np.einsum("oij,oi->oj", blk["W"], dc[cam_idx]), P)
    return np.einsum("pij,pj->pi", Vinv, -blk["gp"] - z)


def model_reduction(blk, dc, dp, cam_idx, pt_idx):
    """Delta L = -g^T Delta - 1/2 sum_k w_k |Jc_k dc_c(k) + Jp_k dp_p(k)|^2.

    The decrease the Gauss-Newton model predicts for the step; it does not
    assume the linear system was solved exactly."""
    JD = np.einsum("oai,oi->oa", blk["Jc"], dc[cam_idx]) + \
        np.einsum("oai,oi->oa", blk["Jp"], dp[pt_idx])
    quad = float(np.sum(blk["w"] * np.sum(JD * JD, axis=1)))
    lin = float(np.sum(blk["gc"] * dc)) + float(np.sum(blk["gp"] * dp))
    return -lin - 0.5 * quad


def _mask_blocks(A, m):
    """Restrict 9x9 blocks to the free parameters: m A m + (I - m)."""
    mm = m[:, :, None] * m[:, None, :]
    return A * mm + np.eye(9)[None] * (1.0 - m)[:, :, None]


def solve_damped(blk, cam_idx, pt_idx, lam, opts, fixed=None):
    """One damped solve (Eq. 2) through the reduced camera system.

    fixed: optional [C, 9] boolean mask of frozen camera parameters.  The
    solve is then the one of the system restricted to the free parameters
    (frozen steps are exactly zero): S -> m S m + (I - m), b -> m b."""
    Us = _ustar(blk["U"], lam, opts.diag_min, opts.diag_max)
    Vinv = point_damped_inverse(blk["V"], lam, opts.diag_min, opts.diag_max)
    C = Us.shape[0]
    m = np.ones((C, 9)) if fixed is None else 1.0 - np.asarray(fixed, dtype=np.float64)
    if opts.solver == "cholesky":
        S, b, _, _ = schur_explicit(blk, cam_idx, pt_idx, lam, opts.diag_min, opts.diag_max)
        mv = m.reshape(-1)
        S = S * mv[:, None] * mv[None, :] + np.diag(1.0 - mv)
        dc = cholesky_solve(S, b * mv).reshape(C, 9)
        its, rel = 0, 0.0
    else:
        b = m * (-blk["gc"] + segment_sum(
            cam_idx, np.einsum("oij,oj->oi", blk["W"],
                               np.einsum("pij,pj->pi", Vinv, blk["gp"])[pt_idx]), C))
        Sii = Us - segment_sum(cam_idx, blk["W"] @ Vinv[pt_idx] @ np.transpose(blk["W"], (0, 2, 1)), C)
        M = np.linalg.inv(_mask_blocks(Sii, m))
        dc, its, rel = pcg(
            lambda x: m * schur_matvec(x, Us, Vinv, blk["W"], cam_idx, pt_idx),
            lambda r: np.einsum("cij,cj->ci", M, r), b, opts.pcg_tol, opts.pcg_maxiter)
    dp = back_substitute(dc, blk, Vinv, cam_idx, pt_idx)
    return dc, dp, its, rel


def dense_lm_delta(cams, points, cam_idx, pt_idx, pixels, lam, delta=0.0,
                   diag_min=1e-6, diag_max=1e32):
    """Eq. 2 written out densely: (H + lambda clamp(diag H)) Delta = -g,
    H = J^T J, g = J^T r with the weighted J; returns (dc [C,9], dp [P,3])."""
    C = np.asarray(cams).shape[0]
    J, rw = dense_jacobian(cams, points, cam_idx, pt_idx, pixels, delta)
    H = J.T @ J
    g = J.T @ rw
    Hs = H + np.diag(damp_diag(np.diag(H), lam, diag_min, diag_max))
    d = np.linalg.solve(Hs, -g)
    return d[:9 * C].reshape(C, 9), d[9 * C:].reshape(-1, 3)


# --------------------------------------------------------------------------
# The LM loop (Alg. 1) with the trust-region damping strategy
# --------------------------------------------------------------------------

@dataclasses.dataclass
class LMOptions:
    """Constants of the LM loop.  up/down are the minimum code example's
    TrustRegion(up=2.0, down=0.5**4); PCG's defaults are its PCG(tol=1e-4,
    maxiter=250).  lambda0, the gain-ratio thresholds and the clamp bounds are
    readings (the paper gives none)."""
    lambda0: float = 1e-4
    up: float = 2.0
    down: float = 0.5 ** 4
    rho_good: float = 0.75
    rho_bad: float = 0.25
    lambda_min: float = 1e-16
    lambda_max: float = 1e32
    diag_min: float = 1e-6
    diag_max: float = 1e32
    solver: str = "pcg"          # "pcg" or "cholesky"
    pcg_tol: float = 1e-4
    pcg_maxiter: int = 250
    huber_delta: float = 0.0


def lm(cams0, points0, cam_idx, pt_idx, pixels, iters, opts=None, fixed=None):
    """Run ``iters`` LM trials (a rejected trial counts as one).

    Per trial: linearise at theta (skipped after a rejection: theta and J are
    unchanged), damp, solve, evaluate F(theta + Delta) and the model
    reduction, gain ratio rho = (F - F') / Delta L.  Accept when F' is finite,
    Delta L > 0 and F' < F.  lambda <- max(lambda/up, lambda_min) when
    accepted with rho > rho_good; lambda <- min(lambda/down, lambda_max) when
    rejected or rho < rho_bad; unchanged otherwise.
    fixed: optional [C, 9] mask of camera parameters that never move.
    Returns (cams, points, trace) with one dict per trial."""
    opts = opts or LMOptions()
    cams = np.array(cams0, dtype=np.float64, copy=True)
    points = np.array(points0, dtype=np.float64, copy=True)
    delta = opts.huber_delta
    lam = opts.lambda0
    F = cost(cams, points, cam_idx, pt_idx, pixels, delta)
    blk = None
    trace = []
    for _ in range(iters):
        if blk is None:
            blk = assemble(cams, points, cam_idx, pt_idx, pixels, delta)
        dc, dp, its, rel = solve_damped(blk, cam_idx, pt_idx, lam, opts, fixed)
        cams_t = cams + dc
        points_t = points + dp
        Ft = cost(cams_t, points_t, cam_idx, pt_idx, pixels, delta)
        dL = model_reduction(blk, dc, dp, cam_idx, pt_idx)
        rho = (F - Ft) / dL if dL != 0.0 else float("nan")
        accept = bool(np.isfinite(Ft) and dL > 0.0 and Ft < F)
        trace.append(dict(cost=F, cost_trial=Ft, model=dL, rho=rho, lam=lam,
                          accepted=accept, pcg_iters=its, pcg_rel_res=rel))
        if accept:
            cams, points, F = cams_t, points_t, Ft
            blk = None
            if rho > opts.rho_good:
                lam = max(lam / opts.up, opts.lambda_min)
            elif rho < opts.rho_bad:
                lam = min(lam / opts.down, opts.lambda_max)
        else:
            lam = min(lam / opts.down, opts.lambda_max)
    return cams, points, trace


# --------------------------------------------------------------------------
# Helpers for tests
# --------------------------------------------------------------------------

def gauge_transform(cams, points, s, Q, tau):
    """Apply the similarity X' = s Q X + tau to a scene.

    Cameras become R' = R Q^T, t' = s t - R Q^T tau, so that
    X'_cam = s X_cam and every projection is unchanged.  omega' is recovered
    with scipy's rotation-vector conversion (a library routine)."""
    from scipy.spatial.transform import Rotation
    cams = np.asarray(cams, dtype=np.float64)
    R = rodrigues(cams[:, 0:3])
    Rn = R @ Q.T
    out = cams.copy()
    out[:, 0:3] = Rotation.from_matrix(Rn).as_rotvec()
    out[:, 3:6] = s * cams[:, 3:6] - np.einsum("cij,j->ci", Rn, tau)
    pts = s * (np.asarray(points, np.float64) @ Q.T) + tau
    return out, pts


def gauge_mask(C):
    """Frozen parameters that remove the 7-dim similarity gauge: all nine of
    camera 0 and the x-translation of camera 1 (scale)."""
    m = np.zeros((C, 9), dtype=bool)
    m[0, :] = True
    if C > 1:
        m[1, 3] = True
    return m


def adjoint_dense(cams, points, cam_idx, pt_idx, pixels, dL_dcams, dL_dpoints, fixed,
                  delta=0.0, lam=0.0, diag_min=1e-6, diag_max=1e32):
    """Implicit-function adjoint at a converged solution, written out densely.

    At the minimiser g(theta*, x) = 0, with the Gauss-Newton H = J^T W J
    restricted to the free parameters f:  v_f = H_ff^{-1} dL/dtheta_f,
    v_fixed = 0;  dL/dx_k = w_k J_k v  (r_k = pi_k - x_k);  for a frozen
    parameter dL/dtheta0 = dL/dtheta - (H v), and 0 for a free one.  lam adds
    lam * clamp(diag H) to H (0: the undamped adjoint).
    Returns (dL/dpixels [O, 2], dL/dcams0 [C, 9], dL/dpoints0 [P, 3], v)."""
    C = np.asarray(cams).shape[0]
    J, _ = dense_jacobian(cams, points, cam_idx, pt_idx, pixels, delta)
    r = residuals(cams, points, cam_idx, pt_idx, pixels)
    _, w = huber(np.sum(r * r, axis=1), delta)
    H = J.T @ J
    H = H + np.diag(damp_diag(np.diag(H), lam, diag_min, diag_max))
    a = np.concatenate([np.asarray(dL_dcams, np.float64).reshape(-1),
                        np.asarray(dL_dpoints, np.float64).reshape(-1)])
    free = np.concatenate([~np.asarray(fixed).reshape(-1), np.ones(a.shape[0] - 9 * C, bool)])
    v = np.zeros_like(a)
    v[free] = np.linalg.solve(H[np.ix_(free, free)], a[free])
    Jv = (J @ v).reshape(-1, 2)                      # sqrt(w) J_k v
    dpix = np.sqrt(w)[:, None] * Jv
    d0 = np.where(free, 0.0, a - H @ v)
    return dpix, d0[:9 * C].reshape(C, 9), d0[9 * C:].reshape(-1, 3), v


def adjoint_schur(cams, points, cam_idx, pt_idx, pixels, dL_dcams, dL_dpoints, fixed,
                  delta=0.0, lam=0.0, diag_min=1e-6, diag_max=1e32):
    """The same adjoint through the Schur complement of the point blocks
    (explicit S, dense Cholesky), for scenes too large for the dense H:
    S v_c = a_c - W V^{-1} a_p,  v_p = V^{-1} (a_p - W^T v_c)."""
    C = np.asarray(cams).shape[0]
    blk = assemble(cams, points, cam_idx, pt_idx, pixels, delta)
    a_c = np.asarray(dL_dcams, np.float64)
    a_p = np.asarray(dL_dpoints, np.float64)
    adj = dict(blk)
    adj["gc"] = -a_c
    adj["gp"] = -a_p
    opts = LMOptions(solver="cholesky", diag_min=diag_min, diag_max=diag_max)
    v_c, v_p, _, _ = solve_damped(adj, cam_idx, pt_idx, lam, opts, fixed)
    sw = np.sqrt(blk["w"])
    Jv = np.einsum("oai,oi->oa", blk["Jc"], v_c[cam_idx]) + \
        np.einsum("oai,oi->oa", blk["Jp"], v_p[pt_idx])
    dpix = (sw * sw)[:, None] * Jv
    Hv_c = segment_sum(cam_idx, blk["w"][:, None] * np.einsum("oai,oa->oi", blk["Jc"], Jv), C)
    if lam > 0.0:
        idx = np.arange(9)
        Hv_c = Hv_c + damp_diag(blk["U"][:, idx, idx], lam, diag_min, diag_max) * v_c
    d0c = np.where(np.asarray(fixed), a_c - Hv_c, 0.0)
    return dpix, d0c, np.zeros_like(a_p), (v_c, v_p)


def pixels_from_scene(scene):
    """Observed pixels: the oracle's projection of the ground truth + noise."""
    return project(scene.cams_gt, scene.points_gt, scene.cam_idx,
                   scene.pt_idx) + scene.noise
