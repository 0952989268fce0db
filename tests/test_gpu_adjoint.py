"""f3: frozen parameters and the implicit-function adjoint (ba_backward)
against the oracle's Schur adjoint, finite differences of GPU re-solves, and
the torch.autograd.Function wrapper."""
import numpy as np
import pytest
import torch

import oracle as orc
import paper_2409_12190_gb300 as ba
import scenegen
from gpu_helpers import np64, problem, rel_err

pytestmark = pytest.mark.gpu


def _converged(sc, pix, prec="f64", jac="auto", trials=30, **kw):
    prob = problem(sc, pix, prec, pcg_maxiter=kw.pop("pcg_maxiter", 600), pcg_tol=kw.pop("pcg_tol", 1e-12),
                   lambda0=1e-6, jacobian=jac, **kw)
    prob.set_fixed(torch.from_numpy(orc.gauge_mask(sc.C)))
    prob.solve(trials)
    torch.cuda.synchronize()
    return prob


def test_frozen_parameters_forward_matches_oracle():
    sc = scenegen.ring_scene(12, 400, seed=31, view_p=0.3)
    pix = orc.pixels_from_scene(sc)
    fixed = orc.gauge_mask(sc.C)
    iters = 8
    c_ref, _, ref = orc.lm(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, iters,
                           orc.LMOptions(solver="cholesky"), fixed=fixed)
    with problem(sc, pix, "f64", pcg_maxiter=9 * sc.C * 3, pcg_tol=1e-14) as prob:
        prob.set_fixed(torch.from_numpy(fixed))
        prob.solve(iters)
        gpu = prob.stats()
        cams, _ = prob.params()
    for g, r in zip(gpu, ref):
        assert abs(g["cost_trial"] - r["cost_trial"]) < 1e-9 * r["cost"]
    assert np.array_equal(np64(cams)[fixed], sc.cams_init[fixed])


@pytest.mark.parametrize("jac", ["store", "recompute"])
@pytest.mark.parametrize("small", [True, False])
def test_backward_matches_oracle_adjoint(jac, small):
    """dL/dpixels and dL/dtheta0 at the GPU's converged parameters equal the
    oracle's Schur + Cholesky adjoint evaluated at the same parameters."""
    sc = scenegen.config_scene("ba64", small=small)
    pix = orc.pixels_from_scene(sc)
    fixed = orc.gauge_mask(sc.C)
    prob = _converged(sc, pix, jac=jac)
    try:
        cams, pts = (np64(t) for t in prob.params())
        rng = np.random.default_rng(3)
        a_c = rng.normal(size=(sc.C, 9))
        a_p = rng.normal(size=(sc.P, 3))
        lam = 1e-6
        dpix, dc0, dp0, its, rel = prob.backward(torch.from_numpy(a_c), torch.from_numpy(a_p), lam=lam,
                                                 maxiter=4000, tol=1e-13)
        ref_pix, ref_c0, ref_p0, _ = orc.adjoint_schur(cams, pts, sc.cam_idx, sc.pt_idx, pix, a_c, a_p,
                                                       fixed, 0.0, lam)
        assert rel < 1e-10, (its, rel)
        assert rel_err(np64(dpix), ref_pix) < 1e-7
        assert rel_err(np64(dc0), ref_c0) < 1e-7
        assert np.all(np64(dc0)[~fixed] == 0.0) and np.all(np64(dp0) == 0.0)
    finally:
        prob.close()


def test_backward_f32_matches_oracle():
    """An FP32 problem's adjoint is solved in FP64 (ba_backward builds an
    FP64 copy of the problem: the system cancels by |U* v| / |S v| ~ 190 and
    has condition ~5.5e3 after block-Jacobi scaling, which would amplify FP32
    rounding to ~1e-2).  It equals the oracle's adjoint at the FP32
    parameters and the FP32-rounded pixels, as the FP64 path does (1e-7),
    on two calls in a row (the second refreshes the FP64 copy)."""
    sc = scenegen.config_scene("ba64", small=True)
    pix = orc.pixels_from_scene(sc)
    pix32 = pix.astype(np.float32).astype(np.float64)
    fixed = orc.gauge_mask(sc.C)
    prob = _converged(sc, pix, prec="f32", pcg_maxiter=400, pcg_tol=1e-6)
    try:
        for call in range(2):
            cams, pts = (np64(t) for t in prob.params())
            a_c = np.zeros((sc.C, 9))
            a_c[:, 3:6] = 2.0 * (cams[:, 3:6] - sc.cams_gt[:, 3:6])
            lam = 1e-4
            dpix, dc0, _, its, rel = prob.backward(torch.from_numpy(a_c), None, lam=lam, maxiter=4000, tol=1e-13)
            assert dpix.dtype == torch.float32
            assert rel < 1e-10, (its, rel)
            ref_pix, ref_c0, _, _ = orc.adjoint_schur(cams, pts, sc.cam_idx, sc.pt_idx, pix32, a_c,
                                                      np.zeros((sc.P, 3)), fixed, 0.0, lam)
            # FP32 outputs: the FP64 adjoint rounded once
            assert rel_err(np64(dpix), ref_pix) < 1e-6
            assert rel_err(np64(dc0), ref_c0) < 1e-6
            if call == 0:
                prob.solve(2)  # move the parameters before the second call
    finally:
        prob.close()


def test_backward_matches_finite_differences_of_gpu_resolves():
    sc = scenegen.ring_scene(6, 60, seed=33, view_p=0.4, noise_px=1e-3)
    pix = orc.pixels_from_scene(sc)
    prob = _converged(sc, pix, trials=40, pcg_maxiter=200, pcg_tol=1e-14)
    try:
        cams, pts = prob.params()
        tgt = torch.tensor(sc.cams_gt[:, 3:6], device="cuda")

        def L(c):
            return float(((c[:, 3:6] - tgt) ** 2).sum())

        g = torch.zeros_like(cams)
        g[:, 3:6] = 2.0 * (cams[:, 3:6] - tgt)
        dpix, _, _, _, _ = prob.backward(g, None, lam=0.0, maxiter=400, tol=1e-14)
        dpix = np64(dpix)
        rng = np.random.default_rng(5)
        h = 1e-5
        for k in rng.choice(sc.O, size=5, replace=False):
            for a in range(2):
                vals = []
                for sgn in (1.0, -1.0):
                    px2 = pix.copy()
                    px2[k, a] += sgn * h
                    prob.set_params(cams, pts)
                    prob.set_pixels(torch.from_numpy(px2).cuda())
                    prob.set_lambda(1e-6)
                    prob.solve(8)
                    vals.append(L(prob.params()[0]))
                fd = (vals[0] - vals[1]) / (2 * h)
                assert abs(fd - dpix[k, a]) < 2e-3 * np.max(np.abs(dpix)) + 1e-9, (k, a, fd, dpix[k, a])
    finally:
        prob.close()


def test_autograd_function_gives_backward():
    sc = scenegen.ring_scene(8, 150, seed=34, view_p=0.35)
    pix = torch.from_numpy(orc.pixels_from_scene(sc)).cuda().requires_grad_(True)
    cams0 = torch.from_numpy(sc.cams_init).cuda().requires_grad_(True)
    pts0 = torch.from_numpy(sc.points_init).cuda().requires_grad_(True)
    prob = problem(sc, pix.detach().cpu().numpy(), "f64", pcg_maxiter=300, pcg_tol=1e-12, lambda0=1e-6)
    prob.set_fixed(torch.from_numpy(orc.gauge_mask(sc.C)))
    try:
        cams, pts = ba.bundle_adjust(pix, cams0, pts0, prob, 25, lam=1e-8, maxiter=600, tol=1e-13)
        tgt = torch.from_numpy(sc.cams_gt[:, 3:6]).cuda()
        loss = ((cams[:, 3:6] - tgt) ** 2).sum()
        gp, gc0, gq0 = torch.autograd.grad(loss, (pix, cams0, pts0))
        g = torch.zeros_like(cams)
        g[:, 3:6] = 2.0 * (cams.detach()[:, 3:6] - tgt)
        dpix, dc0, dp0, _, _ = prob.backward(g, None, lam=1e-8, maxiter=600, tol=1e-13)
        assert torch.allclose(gp, dpix, rtol=1e-9, atol=1e-12 * float(dpix.abs().max()))
        assert torch.allclose(gc0, dc0, rtol=1e-9, atol=1e-12 * float(dc0.abs().max() + 1e-30))
        assert float(gq0.abs().max()) == 0.0
        assert float(gp.abs().max()) > 0.0
    finally:
        prob.close()
