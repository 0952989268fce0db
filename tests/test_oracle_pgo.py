"""Pins of the pose-graph oracle (Sec. IV-D, Eqs. 3-4) against what the
mathematics fixes: closed forms and library routines for Exp / Log (scipy's
expm, logm and rotation vectors), the conjugation identity of Ad, central
differences for the left Jacobian, the edge Jacobian and the gradient, dense
products for the normal equations, Cholesky for the PCG solve, and the zero
minimum of a noise-free graph."""
import numpy as np
import pytest
import scipy.linalg as sl
from scipy.spatial.transform import Rotation

import scenegen
from oracle import LMOptions, left_jacobian
from oracle import pgo

RNG = np.random.default_rng(7)


def _rand_xi(rng, rot=1.0, trans=2.0):
    phi = rng.normal(size=3)
    phi *= rot * rng.uniform(0.05, 1.0) / np.linalg.norm(phi)
    return np.concatenate([rng.normal(size=3) * trans, phi])


def _rand_T(rng):
    return pgo.se3_exp(_rand_xi(rng, rot=2.5, trans=3.0))


def _small_graph(noise=True, full_info=True, seed=3):
    g = scenegen.sphere_graph(4, 6, seed=seed, radius=5.0, full_info=full_info, name="tiny")
    if not noise:
        g.noise[:] = 0.0
    return g


def test_exp_matches_closed_forms():
    rng = np.random.default_rng(1)
    rho = rng.normal(size=3)
    T = pgo.se3_exp(np.concatenate([rho, np.zeros(3)]))
    assert np.allclose(T[:3, :3], np.eye(3), atol=1e-15) and np.allclose(T[:3, 3], rho, atol=1e-14)
    for _ in range(5):
        xi = _rand_xi(rng, rot=3.0)
        T = pgo.se3_exp(xi)
        assert np.allclose(T[:3, :3], Rotation.from_rotvec(xi[3:]).as_matrix(), atol=1e-13)
        # the translation of Exp(rho, phi) is the SO(3) left Jacobian times rho
        assert np.allclose(T[:3, 3], left_jacobian(xi[3:]) @ xi[:3], atol=1e-12)
        assert np.allclose(T[3], [0, 0, 0, 1])


def test_log_inverts_exp_and_matches_logm():
    rng = np.random.default_rng(2)
    for _ in range(10):
        xi = _rand_xi(rng, rot=3.0)
        assert np.allclose(pgo.se3_log(pgo.se3_exp(xi)), xi, atol=1e-11)
        T = _rand_T(rng)
        L = sl.logm(T)
        assert np.allclose(np.imag(L), 0.0, atol=1e-10)
        assert np.allclose(pgo.se3_log(T), pgo.vee6(np.real(L)), atol=1e-10)
    # small angles: the log is the tangent vector
    xi = np.array([0.3, -0.2, 0.1, 1e-9, -2e-9, 3e-9])
    assert np.allclose(pgo.se3_log(pgo.se3_exp(xi)), xi, atol=1e-15)


def test_adjoint_and_bracket_by_their_identities():
    rng = np.random.default_rng(3)
    for _ in range(5):
        T = _rand_T(rng)
        xi = _rand_xi(rng)
        # T Exp(xi) T^-1 = Exp(Ad(T) xi)
        assert np.allclose(T @ pgo.se3_exp(xi) @ pgo.se3_inv(T), pgo.se3_exp(pgo.adjoint(T) @ xi), atol=1e-11)
        # Ad(Exp(xi)) = expm(ad(xi))
        assert np.allclose(pgo.adjoint(pgo.se3_exp(xi)), sl.expm(pgo.ad(xi)), atol=1e-11)
        assert np.allclose(pgo.se3_inv(T) @ T, np.eye(4), atol=1e-13)


def test_left_jacobian_se3():
    rng = np.random.default_rng(4)
    assert np.allclose(pgo.left_jacobian_se3(np.zeros(6)), np.eye(6), atol=1e-15)
    # a pure rotation: both diagonal blocks are the SO(3) left Jacobian
    phi = rng.normal(size=3)
    Jr = pgo.left_jacobian_se3(np.concatenate([np.zeros(3), phi]))
    Jso3 = left_jacobian(phi)
    assert np.allclose(Jr[:3, :3], Jso3, atol=1e-13) and np.allclose(Jr[3:, 3:], Jso3, atol=1e-13)
    assert np.allclose(Jr[:3, 3:], 0.0, atol=1e-13) and np.allclose(Jr[3:, :3], 0.0, atol=1e-15)
    for _ in range(4):
        xi = _rand_xi(rng, rot=2.0)
        J = pgo.left_jacobian_se3(xi)
        # Exp(xi + d) = Exp(J_l(xi) d) Exp(xi) + O(|d|^2): central differences
        h = 1e-6
        Jfd = np.zeros((6, 6))
        Xinv = pgo.se3_inv(pgo.se3_exp(xi))
        for k in range(6):
            e = np.zeros(6)
            e[k] = h
            Jfd[:, k] = (pgo.se3_log(pgo.se3_exp(xi + e) @ Xinv) - pgo.se3_log(pgo.se3_exp(xi - e) @ Xinv)) / (2 * h)
        assert np.allclose(J, Jfd, atol=1e-8)
        # J_l(xi) = Ad(Exp(xi)) J_l(-xi)
        assert np.allclose(J, pgo.adjoint(pgo.se3_exp(xi)) @ pgo.left_jacobian_se3(-xi), atol=1e-11)


def test_edge_jacobian_matches_central_differences():
    rng = np.random.default_rng(5)
    for _ in range(6):
        Ti, Tj = _rand_T(rng), _rand_T(rng)
        # a measurement near the edge's relative pose (residual up to ~1 rad)
        Tm = pgo.se3_exp(_rand_xi(rng, rot=1.0, trans=0.5)) @ pgo.se3_inv(Ti) @ Tj
        A = pgo.edge_jacobian(Ti, Tj, Tm)
        h = 1e-6
        for k in range(6):
            e = np.zeros(6)
            e[k] = h
            dj = (pgo.residual(Ti, pgo.se3_exp(e) @ Tj, Tm) - pgo.residual(Ti, pgo.se3_exp(-e) @ Tj, Tm)) / (2 * h)
            di = (pgo.residual(pgo.se3_exp(e) @ Ti, Tj, Tm) - pgo.residual(pgo.se3_exp(-e) @ Ti, Tj, Tm)) / (2 * h)
            assert np.allclose(A[:, k], dj, atol=2e-7)
            assert np.allclose(-A[:, k], di, atol=2e-7)


def test_residual_is_minus_the_noise_and_cost_is_gauge_invariant():
    g = _small_graph()
    Ts, Tms, infos, Tg = pgo.graph_inputs(g)
    r = pgo.residuals(Tg, g.ei, g.ej, Tms)
    assert np.allclose(r, -g.noise, atol=1e-12)
    G = _rand_T(np.random.default_rng(6))
    F = pgo.cost(Ts, g.ei, g.ej, Tms, infos)
    assert abs(pgo.cost(np.stack([G @ T for T in Ts]), g.ei, g.ej, Tms, infos) - F) <= 1e-9 * F


def test_normal_equations_equal_dense_products():
    g = _small_graph()
    Ts, Tms, infos, _ = pgo.graph_inputs(g)
    blk = pgo.assemble(Ts, g.ei, g.ej, Tms, infos)
    J = pgo.dense_jacobian(blk)
    Om = sl.block_diag(*infos)
    r = blk["r"].reshape(-1)
    H = J.T @ Om @ J
    assert np.allclose(pgo.hessian_dense(blk), H, rtol=1e-12, atol=1e-9 * np.abs(H).max())
    assert np.allclose(blk["g"].reshape(-1), J.T @ Om @ r, atol=1e-9 * np.abs(J.T @ Om @ r).max())
    for n in range(g.N):
        assert np.allclose(blk["Hd"][n], H[6 * n:6 * n + 6, 6 * n:6 * n + 6], atol=1e-9 * np.abs(H).max())
    x = RNG.normal(size=(g.N, 6))
    assert np.allclose(pgo.matvec(blk, x).reshape(-1), H @ x.reshape(-1), atol=1e-9 * np.abs(H).max())


def test_gradient_is_the_derivative_of_the_cost():
    g = _small_graph()
    Ts, Tms, infos, _ = pgo.graph_inputs(g)
    blk = pgo.assemble(Ts, g.ei, g.ej, Tms, infos)
    h = 1e-6
    for n in (0, 5, g.N - 1):
        for k in range(6):
            d = np.zeros((g.N, 6))
            d[n, k] = h
            Fp = pgo.cost(pgo.retract(Ts, d), g.ei, g.ej, Tms, infos)
            Fm = pgo.cost(pgo.retract(Ts, -d), g.ei, g.ej, Tms, infos)
            fd = (Fp - Fm) / (2 * h)
            assert abs(fd - blk["g"][n, k]) <= 1e-5 * max(1.0, abs(blk["g"][n, k])), (n, k, fd, blk["g"][n, k])


def test_model_reduction_is_the_gauss_newton_model():
    g = _small_graph()
    Ts, Tms, infos, _ = pgo.graph_inputs(g)
    blk = pgo.assemble(Ts, g.ei, g.ej, Tms, infos)
    d = RNG.normal(size=(g.N, 6)) * 1e-2
    J = pgo.dense_jacobian(blk)
    Om = sl.block_diag(*infos)
    r = blk["r"].reshape(-1)
    Jd = J @ d.reshape(-1)
    # 1/2 |r|^2 - 1/2 |r + J d|^2 in the Omega metric
    want = 0.5 * r @ Om @ r - 0.5 * (r + Jd) @ Om @ (r + Jd)
    assert abs(pgo.model_reduction(blk, d) - want) <= 1e-10 * abs(r @ Om @ r)


def test_pcg_equals_cholesky_and_fixed_nodes_stay():
    g = _small_graph()
    Ts, Tms, infos, _ = pgo.graph_inputs(g)
    blk = pgo.assemble(Ts, g.ei, g.ej, Tms, infos)
    fixed = np.zeros(g.N, bool)
    fixed[[0, 7]] = True
    dc, _, _ = pgo.solve_damped(blk, 1e-3, LMOptions(solver="cholesky"), fixed)
    dp, its, rel = pgo.solve_damped(blk, 1e-3, LMOptions(solver="pcg", pcg_tol=1e-13, pcg_maxiter=500), fixed)
    assert rel <= 1e-13 and its > 5
    assert np.allclose(dp, dc, atol=1e-9 * np.abs(dc).max())
    assert np.all(dc[fixed] == 0.0) and np.all(dp[fixed] == 0.0)
    # the free rows solve the damped system
    H = pgo.hessian_dense(blk) + np.diag(pgo.damping(blk, 1e-3, LMOptions()).reshape(-1))
    keep = np.repeat(~fixed, 6)
    res = H[np.ix_(keep, keep)] @ dc.reshape(-1)[keep] + blk["g"].reshape(-1)[keep]
    assert np.max(np.abs(res)) <= 1e-9 * np.abs(blk["g"]).max()


def test_lm_reaches_the_zero_minimum_of_a_noise_free_graph():
    g = _small_graph(noise=False)
    Ts, Tms, infos, Tg = pgo.graph_inputs(g)
    fixed = np.zeros(g.N, bool)
    fixed[0] = True  # node 0 carries no drift: the gauge is the truth's
    T, trace = pgo.lm(Ts, g.ei, g.ej, Tms, infos, 12, LMOptions(solver="cholesky"), fixed)
    F0 = trace[0]["cost"]
    assert F0 > 1.0
    assert pgo.cost(T, g.ei, g.ej, Tms, infos) < 1e-16 * F0
    assert np.allclose(T, Tg, atol=1e-7)


@pytest.mark.parametrize("which,N,E", [("sphere2500", 2500, 9799), ("garage1661", 1661, 6275), ("sphere100", 100, None)])
def test_pose_graph_configs_have_the_stated_shapes(which, N, E):
    g = scenegen.pose_graph_config(which)
    assert g.N == N and (E is None or g.E == E)
    assert np.all(g.ei < g.ej) or np.all(g.ei != g.ej)
    assert g.ei.min() >= 0 and g.ej.max() < g.N
    q = g.poses_gt[:, 3:]
    assert np.allclose(np.sum(q * q, 1), 1.0)
    # every information matrix is symmetric positive definite
    for u in g.info[:50]:
        assert np.all(np.linalg.eigvalsh(pgo.info_matrix(u)) > 0)
