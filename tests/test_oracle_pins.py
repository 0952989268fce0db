"""Pins for the FP64 oracle: checks against mathematics that does not come
from the oracle itself (closed forms, library routines, finite differences,
invariants, brute force).  CPU only."""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle as orc
import scenegen


def _rand_rotvec(rng, theta):
    axis = rng.normal(size=3)
    return theta * axis / np.linalg.norm(axis)


ANGLES = [0.0, 1e-12, 1e-9, 3e-5, 2e-4, 0.05, 0.099, 0.101, 0.3, 1.0, 2.5,
          np.pi - 1e-6]


@pytest.mark.parametrize("theta", ANGLES)
def test_rodrigues_is_matrix_exponential(theta):
    """R(omega) = expm([omega]_x) (scipy's Pade expm, a library routine)."""
    rng = np.random.default_rng(int(theta * 1e6) % 1000 + 7)
    w = _rand_rotvec(rng, theta)
    R = orc.rodrigues(w)
    E = sl.expm(orc.skew(w))
    assert np.max(np.abs(R - E)) < 2e-15
    assert np.max(np.abs(R @ R.T - np.eye(3))) < 2e-15


@pytest.mark.parametrize("theta", ANGLES)
def test_left_jacobian_by_series(theta):
    """J_l(w) = sum_n [w]_x^n / (n+1)!  (its defining power series)."""
    rng = np.random.default_rng(11)
    w = _rand_rotvec(rng, theta)
    K = orc.skew(w)
    S = np.zeros((3, 3))
    term = np.eye(3)
    fact = 1.0
    for n in range(60):
        fact *= (n + 1)
        S += term / fact
        term = term @ K
    assert np.max(np.abs(orc.left_jacobian(w) - S)) < 5e-15


def test_left_jacobian_perturbation_identity():
    """R(w + d) R(w)^T = expm([J_l(w) d]_x) + O(|d|^2), checked by central
    differences of R(w + e d)."""
    rng = np.random.default_rng(3)
    for theta in [1e-7, 0.02, 0.7, 2.9]:
        w = _rand_rotvec(rng, theta)
        d = rng.normal(size=3)
        e = 1e-6
        dR = (orc.rodrigues(w + e * d) - orc.rodrigues(w - e * d)) / (2 * e)
        lhs = dR @ orc.rodrigues(w).T
        rhs = orc.skew(orc.left_jacobian(w) @ d)
        assert np.max(np.abs(lhs - rhs)) < 1e-8


def test_projection_closed_forms():
    """Hand-computed pixels of the BAL camera."""
    cams = np.zeros((3, 9))
    cams[:, 5] = -5.0
    cams[:, 6] = 500.0
    cams[1, 7] = 0.1                       # k1
    cams[2, 1] = np.pi / 2                 # rotation about y by 90 degrees
    pts = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    ci = np.array([0, 1, 2, 2])
    pi = np.array([0, 0, 0, 1])
    out = orc.project(cams, pts, ci, pi)
    # X_cam = (1,0,-5): p = -(1,0)/(-5) = (0.2, 0); pixel 500 * 0.2
    assert np.allclose(out[0], [100.0, 0.0], atol=1e-12)
    # |p|^2 = 0.04, distortion 1 + 0.1 * 0.04
    assert np.allclose(out[1], [100.4, 0.0], atol=1e-12)
    # R_y(pi/2) (1,0,0) = (0,0,-1): X_cam = (0,0,-6), on the optical axis
    assert np.allclose(out[2], [0.0, 0.0], atol=1e-12)
    # R_y(pi/2) (0,0,1) = (1,0,0): X_cam = (1,0,-5)
    assert np.allclose(out[3], [100.0, 0.0], atol=1e-10)


def _random_cameras(rng, n, thetas):
    cams = np.zeros((n, 9))
    for i in range(n):
        cams[i, 0:3] = _rand_rotvec(rng, thetas[i % len(thetas)])
    cams[:, 3:5] = rng.normal(0, 0.5, size=(n, 2))
    cams[:, 5] = -5.0 + rng.normal(0, 0.3, size=n)
    cams[:, 6] = 400.0 + 200.0 * rng.random(n)
    cams[:, 7] = rng.normal(0, 0.05, size=n)
    cams[:, 8] = rng.normal(0, 0.02, size=n)
    return cams


def test_jacobian_matches_central_differences():
    """Analytic Jc, Jp against central differences of the residual, including
    the small-angle branches and a rotation near pi."""
    rng = np.random.default_rng(5)
    thetas = [0.0, 1e-9, 5e-5, 0.05, 0.5, 2.0, np.pi - 1e-4]
    C = len(thetas)
    cams = _random_cameras(rng, C, thetas)
    # points in front of each camera: X = R^T (X_cam - t) with X_cam[2] < 0
    pts, ci, pi = [], [], []
    for i in range(C):
        R = orc.rodrigues(cams[i, 0:3])
        for _ in range(4):
            Xc = np.array([rng.normal(0, 1.0), rng.normal(0, 1.0), -4.0 - 2 * rng.random()])
            pts.append(R.T @ (Xc - cams[i, 3:6]))
            ci.append(i)
            pi.append(len(pts) - 1)
    pts = np.array(pts)
    ci = np.array(ci)
    pi = np.array(pi)
    pix = rng.normal(0, 50, size=(len(ci), 2))
    r, Jc, Jp = orc.linearize(cams, pts, ci, pi, pix)
    assert np.allclose(r, orc.residuals(cams, pts, ci, pi, pix), atol=0, rtol=0)
    for k in range(len(ci)):
        for a in range(9):
            h = 1e-6 * max(1.0, abs(cams[ci[k], a]))
            cp = cams.copy()
            cm = cams.copy()
            cp[ci[k], a] += h
            cm[ci[k], a] -= h
            fd = (orc.residuals(cp, pts, ci[k:k + 1], pi[k:k + 1], pix[k:k + 1]) -
                  orc.residuals(cm, pts, ci[k:k + 1], pi[k:k + 1], pix[k:k + 1]))[0] / (2 * h)
            scale = max(1.0, np.max(np.abs(Jc[k, :, a])))
            assert np.max(np.abs(fd - Jc[k, :, a])) < 2e-6 * scale, (k, a)
        for a in range(3):
            h = 1e-6 * max(1.0, abs(pts[pi[k], a]))
            pp = pts.copy()
            pm = pts.copy()
            pp[pi[k], a] += h
            pm[pi[k], a] -= h
            fd = (orc.residuals(cams, pp, ci[k:k + 1], pi[k:k + 1], pix[k:k + 1]) -
                  orc.residuals(cams, pm, ci[k:k + 1], pi[k:k + 1], pix[k:k + 1]))[0] / (2 * h)
            scale = max(1.0, np.max(np.abs(Jp[k, :, a])))
            assert np.max(np.abs(fd - Jp[k, :, a])) < 2e-6 * scale, (k, a)


def _tiny_scene(seed, C=4, P=12, noise=1.0, delta=0.0, outliers=0.0):
    sc = scenegen.ring_scene(C, P, seed=seed, view_p=0.5, noise_px=noise,
                             outlier_frac=outliers, huber_delta=delta)
    pix = orc.pixels_from_scene(sc)
    return sc, pix


def test_huber_with_large_delta_is_plain_loss():
    sc, pix = _tiny_scene(1)
    a = orc.assemble(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, 0.0)
    b = orc.assemble(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, 1e9)
    for key in ("U", "V", "W", "gc", "gp"):
        assert np.array_equal(a[key], b[key])
    assert a["F"] == b["F"]


def test_huber_closed_form():
    rho, w = orc.huber(np.array([0.25, 1.0, 4.0, 9.0]), 1.0)
    assert np.allclose(rho, [0.25, 1.0, 3.0, 5.0])       # 2*sqrt(s) - 1 outside
    assert np.allclose(w, [1.0, 1.0, 0.5, 1.0 / 3.0])     # rho'(s) = 1/sqrt(s)


@pytest.mark.parametrize("delta,outliers", [(0.0, 0.0), (1.0, 0.3)])
def test_block_assembly_equals_dense(delta, outliers):
    """U, V, W, g from the per-observation blocks equal J^T J and J^T r of the
    dense weighted Jacobian (brute force)."""
    sc, pix = _tiny_scene(2, C=5, P=15, delta=delta, outliers=outliers)
    args = (sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, delta)
    blk = orc.assemble(*args)
    J, rw = orc.dense_jacobian(*args)
    H = J.T @ J
    g = J.T @ rw
    C, P = sc.C, sc.P
    scale = np.max(np.abs(H))
    for i in range(C):
        assert np.max(np.abs(H[9 * i:9 * i + 9, 9 * i:9 * i + 9] - blk["U"][i])) < 1e-13 * scale
        assert np.max(np.abs(g[9 * i:9 * i + 9] - blk["gc"][i])) < 1e-13 * np.max(np.abs(g))
    for j in range(P):
        o = 9 * C + 3 * j
        assert np.max(np.abs(H[o:o + 3, o:o + 3] - blk["V"][j])) < 1e-13 * scale
        assert np.max(np.abs(g[o:o + 3] - blk["gp"][j])) < 1e-13 * np.max(np.abs(g))
    Wsum = np.zeros((C, P, 9, 3))
    for k in range(sc.O):
        Wsum[sc.cam_idx[k], sc.pt_idx[k]] += blk["W"][k]
    for i in range(C):
        for j in range(P):
            o = 9 * C + 3 * j
            assert np.max(np.abs(H[9 * i:9 * i + 9, o:o + 3] - Wsum[i, j])) < 1e-13 * scale
    # camera-camera blocks of H vanish: no residual touches two cameras
    for i in range(C):
        for l in range(C):
            if i != l:
                assert np.all(H[9 * i:9 * i + 9, 9 * l:9 * l + 9] == 0.0)


def test_schur_solve_equals_dense_solve():
    """Schur complement + Cholesky + back-substitution solves the full damped
    system exactly (textbook block elimination), and tight PCG agrees."""
    sc, pix = _tiny_scene(3, C=5, P=20, delta=1.0, outliers=0.2)
    lam = 1e-3
    args = (sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix)
    blk = orc.assemble(*args, 1.0)
    dc_d, dp_d = orc.dense_lm_delta(*args, lam, delta=1.0)
    opts = orc.LMOptions(solver="cholesky", huber_delta=1.0)
    dc, dp, _, _ = orc.solve_damped(blk, sc.cam_idx, sc.pt_idx, lam, opts)
    sc_ = np.max(np.abs(dc_d))
    assert np.max(np.abs(dc - dc_d)) < 1e-9 * sc_
    assert np.max(np.abs(dp - dp_d)) < 1e-9 * max(np.max(np.abs(dp_d)), sc_)
    opts = orc.LMOptions(solver="pcg", pcg_tol=1e-15, pcg_maxiter=9 * sc.C * 4,
                         huber_delta=1.0)
    dc2, dp2, its, rel = orc.solve_damped(blk, sc.cam_idx, sc.pt_idx, lam, opts)
    assert np.max(np.abs(dc2 - dc_d)) < 1e-7 * sc_
    # residual of the full system
    J, rw = orc.dense_jacobian(*args, 1.0)
    H = J.T @ J
    g = J.T @ rw
    Hs = H + np.diag(orc.damp_diag(np.diag(H), lam, 1e-6, 1e32))
    d = np.concatenate([dc.reshape(-1), dp.reshape(-1)])
    assert np.linalg.norm(Hs @ d + g) < 1e-10 * np.linalg.norm(g)


def test_implicit_schur_matvec_and_block_jacobi():
    sc, pix = _tiny_scene(4, C=6, P=25)
    lam = 1e-2
    blk = orc.assemble(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix)
    S, b, Us, Vinv = orc.schur_explicit(blk, sc.cam_idx, sc.pt_idx, lam)
    rng = np.random.default_rng(0)
    x = rng.normal(size=(sc.C, 9))
    Sx = orc.schur_matvec(x, Us, Vinv, blk["W"], sc.cam_idx, sc.pt_idx)
    assert np.max(np.abs(Sx.reshape(-1) - S @ x.reshape(-1))) < 1e-11 * np.max(np.abs(S @ x.reshape(-1)))
    M = orc.block_jacobi(Us, Vinv, blk["W"], sc.cam_idx, sc.pt_idx)
    for i in range(sc.C):
        Sii = S[9 * i:9 * i + 9, 9 * i:9 * i + 9]
        assert np.max(np.abs(M[i] @ Sii - np.eye(9))) < 1e-8
    assert np.all(np.linalg.eigvalsh(S) > 0)


def test_pcg_terminates_in_n_steps_on_spd():
    """CG on an SPD n x n system reaches the solution in at most n steps
    (exact arithmetic); checked against numpy's dense solve."""
    rng = np.random.default_rng(8)
    n = 30
    Q = rng.normal(size=(n, n))
    A = Q @ Q.T / n + np.diag(np.linspace(0.5, 3.0, n))
    b = rng.normal(size=n)
    Dinv = 1.0 / np.diag(A)
    x, its, rel = orc.pcg(lambda v: A @ v, lambda v: Dinv * v, b, 1e-13, 4 * n)
    assert its <= n
    assert np.max(np.abs(x - np.linalg.solve(A, b))) < 1e-9 * np.max(np.abs(x))
    x1, its1, _ = orc.pcg(lambda v: A @ v, lambda v: Dinv * v, b, 1e-13, 1)
    # one step is the exact line minimisation along the preconditioned gradient
    z = Dinv * b
    assert np.allclose(x1, (b @ z) / (z @ A @ z) * z, rtol=1e-12, atol=0)


def test_model_reduction_closed_form_for_exact_step():
    """With (H + lambda D) Delta = -g solved exactly,
    -g^T Delta - 1/2 Delta^T H Delta = 1/2 (-g^T Delta + lambda Delta^T D Delta)."""
    sc, pix = _tiny_scene(5, C=5, P=20)
    lam = 0.3
    args = (sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix)
    blk = orc.assemble(*args)
    dc, dp, _, _ = orc.solve_damped(blk, sc.cam_idx, sc.pt_idx, lam,
                                    orc.LMOptions(solver="cholesky"))
    dL = orc.model_reduction(blk, dc, dp, sc.cam_idx, sc.pt_idx)
    J, rw = orc.dense_jacobian(*args)
    H = J.T @ J
    g = J.T @ rw
    D = np.clip(np.diag(H), 1e-6, 1e32)
    d = np.concatenate([dc.reshape(-1), dp.reshape(-1)])
    ref = 0.5 * (-(g @ d) + lam * d @ (D * d))
    assert abs(dL - ref) < 1e-10 * abs(ref)
    assert dL > 0


def test_gain_ratio_tends_to_one_for_small_steps():
    sc, pix = _tiny_scene(6, C=4, P=20)
    args = (sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix)
    blk = orc.assemble(*args)
    F = orc.cost(*args)
    for lam, tol in [(1e4, 1e-2), (1e6, 1e-4)]:
        dc, dp, _, _ = orc.solve_damped(blk, sc.cam_idx, sc.pt_idx, lam,
                                        orc.LMOptions(solver="cholesky"))
        Ft = orc.cost(sc.cams_init + dc, sc.points_init + dp, sc.cam_idx, sc.pt_idx, pix)
        dL = orc.model_reduction(blk, dc, dp, sc.cam_idx, sc.pt_idx)
        assert abs((F - Ft) / dL - 1.0) < tol


def test_cost_is_gauge_invariant():
    """F is unchanged by a global similarity applied to cameras and points."""
    sc, pix = _tiny_scene(7, C=6, P=40)
    from scipy.spatial.transform import Rotation
    Q = Rotation.from_rotvec([0.3, -0.2, 0.5]).as_matrix()
    cams2, pts2 = orc.gauge_transform(sc.cams_init, sc.points_init, 1.7, Q,
                                      np.array([0.4, -1.0, 0.25]))
    F1 = orc.cost(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix)
    F2 = orc.cost(cams2, pts2, sc.cam_idx, sc.pt_idx, pix)
    assert abs(F1 - F2) < 1e-11 * F1


def test_jacobian_has_seven_dim_gauge_null_space():
    """At a noise-free solution J has a 7-dimensional null space (rotation,
    translation, scale of the whole scene): the 7 smallest singular values are
    far below the 8th.  A wrong sign or index in Jc/Jp breaks this."""
    sc, _ = _tiny_scene(8, C=5, P=30, noise=0.0)
    pix = orc.project(sc.cams_gt, sc.points_gt, sc.cam_idx, sc.pt_idx)
    J, _ = orc.dense_jacobian(sc.cams_gt, sc.points_gt, sc.cam_idx, sc.pt_idx, pix)
    s = np.linalg.svd(J, compute_uv=False)
    assert s[-7] < 1e-9 * s[0]
    assert s[-8] > 1e-6 * s[0]


def test_noise_free_lm_reaches_zero_cost():
    sc = scenegen.ring_scene(8, 200, seed=9, view_p=0.3, noise_px=0.0)
    pix = orc.pixels_from_scene(sc)
    opts = orc.LMOptions(solver="cholesky")
    _, _, trace = orc.lm(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, 30, opts)
    F0 = trace[0]["cost"]
    Ffinal = min(t["cost_trial"] for t in trace if t["accepted"])
    assert F0 > 1.0
    assert Ffinal < 1e-20 * sc.O


def test_lm_accepted_costs_are_monotone():
    sc = scenegen.config_scene("ba16")
    pix = orc.pixels_from_scene(sc)
    opts = orc.LMOptions(solver="cholesky")
    _, _, trace = orc.lm(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, 8, opts)
    costs = [trace[0]["cost"]] + [t["cost_trial"] for t in trace if t["accepted"]]
    assert all(b <= a for a, b in zip(costs, costs[1:]))
    assert costs[-1] < 0.1 * costs[0]
    # with 1 px noise the converged mean squared error is about 2 sigma^2 * (1 - dof/2O)
    mse = 2.0 * costs[-1] / sc.O
    assert 1.5 < mse < 2.2


def _counting_sort(keys, n):
    counts = [0] * n
    for k in keys:
        counts[k] += 1
    rowptr = [0]
    for c in counts:
        rowptr.append(rowptr[-1] + c)
    cursor = rowptr[:-1].copy()
    perm = [0] * len(keys)
    for i, k in enumerate(keys):
        perm[cursor[k]] = i
        cursor[k] += 1
    return perm, rowptr


@pytest.mark.parametrize("n,O", [(1, 0), (1, 5), (7, 50), (300, 2000), (5000, 3000)])
def test_csr_build_is_stable_counting_sort(n, O):
    rng = np.random.default_rng(n + O)
    keys = rng.integers(0, n, size=O)
    perm, rowptr = orc.csr_build(keys, n)
    p2, r2 = _counting_sort(keys.tolist(), n)
    assert perm.tolist() == p2
    assert rowptr.tolist() == r2


# --------------------------------------------------------------------------
# implicit-function adjoint
# --------------------------------------------------------------------------

def _converge(cams, pts, ci, pi, pix, fixed, iters=40):
    opts = orc.LMOptions(solver="cholesky", lambda0=1e-6)
    c, p, tr = orc.lm(cams, pts, ci, pi, pix, iters, opts, fixed=fixed)
    return c, p, tr


def test_gauge_fixed_lm_keeps_frozen_parameters():
    sc = scenegen.ring_scene(6, 60, seed=21, view_p=0.4, noise_px=1.0)
    pix = orc.pixels_from_scene(sc)
    fixed = orc.gauge_mask(sc.C)
    c, _, tr = _converge(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, fixed, 15)
    assert np.array_equal(c[fixed], sc.cams_init[fixed])
    assert tr[-1]["cost"] < 0.05 * tr[0]["cost"]


def test_adjoint_matches_central_differences():
    """dL/dx from the implicit-function adjoint equals central differences of
    L(theta*(x)) with warm-started re-solves (noise 1e-3 px, where the
    Gauss-Newton Hessian is the exact one up to O(residual))."""
    sc = scenegen.ring_scene(5, 40, seed=22, view_p=0.4, noise_px=1e-3)
    pix = orc.pixels_from_scene(sc)
    fixed = orc.gauge_mask(sc.C)
    ci, pi = sc.cam_idx, sc.pt_idx
    c, p, _ = _converge(sc.cams_init, sc.points_init, ci, pi, pix, fixed, 40)
    tgt = sc.cams_gt[:, 3:6]

    def L(cams):
        return float(np.sum((cams[:, 3:6] - tgt) ** 2))

    dLc = np.zeros_like(c)
    dLc[:, 3:6] = 2.0 * (c[:, 3:6] - tgt)
    dpix, d0c, d0p, _ = orc.adjoint_dense(c, p, ci, pi, pix, dLc, np.zeros_like(p), fixed)
    rng = np.random.default_rng(0)
    h = 1e-5
    for k in rng.choice(sc.O, size=6, replace=False):
        for a in range(2):
            vals = []
            for sgn in (1.0, -1.0):
                px2 = pix.copy()
                px2[k, a] += sgn * h
                c2, _, _ = _converge(c, p, ci, pi, px2, fixed, 8)
                vals.append(L(c2))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - dpix[k, a]) < 1e-3 * np.max(np.abs(dpix)) + 1e-9, (k, a, fd, dpix[k, a])
    # initial values: free parameters do not influence theta*, frozen ones do
    assert np.all(d0c[~fixed] == 0.0) and np.all(d0p == 0.0)
    j = 1  # camera 1's frozen t_x
    e = np.zeros_like(c)
    e[j, 3] = h
    cp, _, _ = _converge(c + e, p, ci, pi, pix, fixed, 8)
    cm, _, _ = _converge(c - e, p, ci, pi, pix, fixed, 8)
    fd0 = (L(cp) - L(cm)) / (2 * h)
    assert abs(fd0 - d0c[j, 3]) < 1e-3 * abs(d0c[j, 3]) + 1e-9


def test_adjoint_schur_equals_dense():
    sc = scenegen.ring_scene(6, 50, seed=23, view_p=0.4, noise_px=1.0, outlier_frac=0.1,
                             huber_delta=1.0)
    pix = orc.pixels_from_scene(sc)
    fixed = orc.gauge_mask(sc.C)
    rng = np.random.default_rng(1)
    a_c = rng.normal(size=(sc.C, 9))
    a_p = rng.normal(size=(sc.P, 3))
    for lam in (0.0, 1e-3):
        d1 = orc.adjoint_dense(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, a_c, a_p,
                               fixed, 1.0, lam)
        d2 = orc.adjoint_schur(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, a_c, a_p,
                               fixed, 1.0, lam)
        for x, y in zip(d1[:3], d2[:3]):
            assert np.max(np.abs(x - y)) <= 1e-8 * max(np.max(np.abs(x)), 1e-30)


@pytest.mark.parametrize("delta", [0.5, 1.0, 3.0])
def test_huber_is_continuous_with_its_derivative_at_delta(delta):
    """rho and rho' (the IRLS weight) meet at |r| = delta: no jump in the
    loss or in the gradient where an observation turns into an outlier."""
    s0 = delta * delta
    eps = 1e-9
    rho, w = orc.huber(np.array([s0 * (1 - eps), s0, s0 * (1 + eps)]), delta)
    assert np.all(np.abs(rho - s0) <= 4 * eps * s0)
    assert np.all(np.abs(w - 1.0) <= 4 * eps)
    # rho'(s) by central differences on the outlier side equals the weight
    s = np.array([2.0, 7.0, 30.0]) * s0
    h = 1e-6 * s
    d = (orc.huber(s + h, delta)[0] - orc.huber(s - h, delta)[0]) / (2 * h)
    assert np.allclose(d, orc.huber(s, delta)[1], rtol=1e-7)


def test_huber_gradient_is_the_gradient_of_the_cost():
    """Under Huber's loss with outliers, the assembled g = sum_k w_k J_k^T r_k
    is the gradient of F = 1/2 sum rho(|r|^2) (central differences of the
    cost alone): this fixes the 1/2, the weight w = rho' and J together."""
    sc, pix = _tiny_scene(31, C=3, P=8, delta=1.0, outliers=0.4)
    args = (sc.cam_idx, sc.pt_idx, pix, sc.huber_delta)
    # at the ground truth the residuals are the 1 px noise and the 20 px
    # outliers, so both regimes of the loss are present
    cams, pts = sc.cams_gt, sc.points_gt
    blk = orc.assemble(cams, pts, sc.cam_idx, sc.pt_idx, pix, sc.huber_delta)
    _, w = orc.huber(np.sum(blk["r"] ** 2, axis=1), sc.huber_delta)
    assert np.any(w < 1.0) and np.any(w == 1.0)
    g = np.concatenate([blk["gc"].reshape(-1), blk["gp"].reshape(-1)])
    theta = np.concatenate([cams.reshape(-1), pts.reshape(-1)])
    nc = cams.size

    def F(t):
        return orc.cost(t[:nc].reshape(cams.shape), t[nc:].reshape(pts.shape), *args)

    num = np.empty_like(theta)
    for i in range(theta.size):
        h = 1e-6 * max(1.0, abs(theta[i]))
        e = np.zeros_like(theta)
        e[i] = h
        num[i] = (F(theta + e) - F(theta - e)) / (2 * h)
    assert np.max(np.abs(num - g)) <= 1e-6 * np.max(np.abs(g))


@pytest.mark.parametrize("seed", range(24))
def test_random_tiny_scenes_blocks_and_schur_solve_equal_dense(seed):
    """Fuzz over random tiny problems (2-5 cameras, 5-30 points, random
    visibility, with or without Huber outliers, random damping): the block
    assembly equals the dense J^T J / J^T r, and the Schur-complement solve
    equals the dense solve of Eq. 2 built from the dense Jacobian."""
    rng = np.random.default_rng(1000 + seed)
    C = int(rng.integers(2, 6))
    P = int(rng.integers(5, 31))
    huber = bool(seed % 2)
    sc = scenegen.arc_scene(C, P, seed=seed, views_lo=min(2, C), views_hi=C,
                            huber_delta=1.0 if huber else 0.0)
    pix = orc.pixels_from_scene(sc)
    if huber:   # a few large residuals so both regimes of the loss occur
        pix = pix + (rng.random((sc.O, 1)) < 0.3) * rng.normal(0.0, 15.0, size=(sc.O, 2))
    lam = float(10.0 ** rng.uniform(-4, 0))
    args = (sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix)
    blk = orc.assemble(*args, sc.huber_delta)
    J, rw = orc.dense_jacobian(*args, sc.huber_delta)
    H = J.T @ J
    g = J.T @ rw
    nc = 9 * C
    for key, ref in (("U", [H[9 * i:9 * i + 9, 9 * i:9 * i + 9] for i in range(C)]),
                     ("V", [H[nc + 3 * j:nc + 3 * j + 3, nc + 3 * j:nc + 3 * j + 3] for j in range(P)])):
        assert np.allclose(blk[key], np.array(ref), rtol=1e-12, atol=1e-12 * np.abs(H).max())
    assert np.allclose(blk["gc"].reshape(-1), g[:nc], rtol=1e-12, atol=1e-12 * np.abs(g).max())
    assert np.allclose(blk["gp"].reshape(-1), g[nc:], rtol=1e-12, atol=1e-12 * np.abs(g).max())
    dc, dp, _, _ = orc.solve_damped(blk, sc.cam_idx, sc.pt_idx, lam, orc.LMOptions(solver="cholesky"))
    dc_ref, dp_ref = orc.dense_lm_delta(*args, lam, sc.huber_delta)
    scale = max(np.abs(dc_ref).max(), np.abs(dp_ref).max())
    assert np.max(np.abs(dc - dc_ref)) <= 1e-8 * scale
    assert np.max(np.abs(dp - dp_ref)) <= 1e-8 * scale
