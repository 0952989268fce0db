"""a6 and the whole LM loop against the oracle: per-trial cost traces (FP64,
1e-9 relative), final parameters (1e-7 of their scale), FP32 final cost
(1e-6 relative), graph replay, determinism, checkpoint / resume."""
import numpy as np
import pytest
import torch

import oracle as orc
import paper_2409_12190_gb300 as ba
import scenegen
from gpu_helpers import np64, problem, small_ring

pytestmark = pytest.mark.gpu


def _trace_rel(gpu, ref, key):
    return max(abs(g[key] - r[key]) / abs(r[key]) for g, r in zip(gpu, ref))


@pytest.mark.parametrize("jac", ["store", "recompute"])
def test_ba16_f64_trace_matches_oracle_cholesky(jac):
    sc = scenegen.config_scene("ba16")
    pix = orc.pixels_from_scene(sc)
    iters = 20
    cams_ref, pts_ref, ref = orc.lm(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix,
                                    iters, orc.LMOptions(solver="cholesky"))
    with problem(sc, pix, "f64", pcg_maxiter=9 * sc.C, pcg_tol=1e-14, jacobian=jac) as prob:
        prob.solve(iters)
        gpu = prob.stats()
        cams, pts = prob.params()
    assert len(gpu) == iters
    assert _trace_rel(gpu, ref, "cost") < 1e-9
    assert _trace_rel(gpu, ref, "cost_trial") < 1e-9
    # decisions agree while the steps are far above rounding level
    for g, r in zip(gpu, ref):
        if abs(r["cost"] - r["cost_trial"]) > 1e-7 * r["cost"]:
            assert g["accepted"] == r["accepted"]
    scale = np.maximum(1.0, np.abs(cams_ref))
    assert np.max(np.abs(np64(cams) - cams_ref) / scale) < 1e-7
    assert np.max(np.abs(np64(pts) - pts_ref) / np.maximum(1.0, np.abs(pts_ref))) < 1e-7


@pytest.mark.parametrize("jac", ["store", "recompute"])
def test_ring_f64_huber_trace_matches_oracle_pcg(jac):
    """Per-trial parity at 1e-9 with PCG truncated where CG's rounding
    amplification is still far below 1e-9 (10 iterations)."""
    sc = small_ring()
    pix = orc.pixels_from_scene(sc)
    iters = 8
    opts = orc.LMOptions(solver="pcg", pcg_tol=1e-4, pcg_maxiter=10, huber_delta=1.0)
    _, _, ref = orc.lm(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, iters, opts)
    with problem(sc, pix, "f64", pcg_maxiter=10, pcg_tol=1e-4, jacobian=jac) as prob:
        prob.solve(iters)
        gpu = prob.stats()
    assert _trace_rel(gpu, ref, "cost") < 1e-9
    assert _trace_rel(gpu, ref, "cost_trial") < 1e-9
    assert [g["pcg_iters"] for g in gpu] == [r["pcg_iters"] for r in ref]
    assert [g["accepted"] for g in gpu] == [r["accepted"] for r in ref]


def test_ring_f64_huber_trace_matches_oracle_pcg_15():
    """The same at 15 PCG iterations per trial, the most at which the
    oracle's own trace on this scene is insensitive to the summation order
    (with the observations permuted its trial costs move by ~3e-13; at 25
    iterations by ~5e-10 and at 50 by ~3e-4: CG on this ring amplifies
    rounding exponentially with the iteration count, so beyond ~20
    iterations no implementation can be compared to 1e-9 on it -- the
    50-iteration setting is compared at full size on ba250, whose reduced
    system is better conditioned, and with exact solves in
    test_gpu_converged)."""
    sc = small_ring()
    pix = orc.pixels_from_scene(sc)
    iters = 8
    opts = orc.LMOptions(solver="pcg", pcg_tol=1e-4, pcg_maxiter=15, huber_delta=1.0)
    _, _, ref = orc.lm(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, iters, opts)
    with problem(sc, pix, "f64", pcg_maxiter=15, pcg_tol=1e-4) as prob:
        prob.solve(iters)
        gpu = prob.stats()
    assert _trace_rel(gpu, ref, "cost") < 1e-9
    assert _trace_rel(gpu, ref, "cost_trial") < 1e-9
    assert [g["pcg_iters"] for g in gpu] == [r["pcg_iters"] for r in ref]
    assert [g["accepted"] for g in gpu] == [r["accepted"] for r in ref]


def _converged_cost(trace):
    acc = [t["cost_trial"] for t in trace if t["accepted"]]
    return min([trace[0]["cost"]] + acc)


def _run_until_stall(prob, cap, window=50, rel=1e-10):
    """LM trials in windows until a window lowers the cost by less than rel
    (relative) or cap trials ran; returns the per-trial costs."""
    costs = []
    while len(costs) < cap:
        prob.solve(window)
        st = prob.stats(cap=window)
        costs += [t["cost_trial"] if t["accepted"] else t["cost"] for t in st]
        if len(costs) > window and costs[-window - 1] - costs[-1] <= rel * costs[-1]:
            break
    return costs


@pytest.mark.parametrize("jac", ["store", "recompute"])
def test_ring_f32_reaches_the_oracles_converged_cost(jac):
    """Plain loss: the LM converges (quadratically) within 25 trials, in
    FP64 on the oracle and in FP32 on the GPU; the FP32 cost, re-evaluated
    in FP64 by the oracle at the returned parameters, is within 1e-6 of the
    oracle's converged cost."""
    sc = small_ring(C=60, P=3000, huber=False)
    pix = orc.pixels_from_scene(sc)
    iters = 25
    opts = orc.LMOptions(solver="pcg", pcg_tol=1e-4, pcg_maxiter=50)
    _, _, ref = orc.lm(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, iters, opts)
    F_ref = _converged_cost(ref)
    # converged: the oracle's last five trials gained nothing measurable
    assert ref[-5]["cost"] - F_ref <= 1e-12 * F_ref
    with problem(sc, pix, "f32", pcg_maxiter=50, pcg_tol=1e-4, jacobian=jac) as prob:
        prob.solve(iters)
        gpu = prob.stats()
        cams, pts = prob.params()
    F32 = _converged_cost(gpu)
    F32_exact = orc.cost(np64(cams), np64(pts), sc.cam_idx, sc.pt_idx, pix)
    assert abs(F32_exact - F_ref) < 1e-6 * F_ref
    assert abs(F32 - F_ref) < 1e-6 * F_ref


@pytest.mark.parametrize("jac", ["store", "recompute"])
def test_ring_huber_f32_converges_to_the_f64_cost(jac):
    """Huber: IRLS without the rho'' term converges only linearly (on the
    outlier residuals the loss is linear and each trial removes a fraction
    of the excess), so both precisions are run until their cost stops
    decreasing; the FP32 cost is then within 1e-6 of the FP64 cost, whose
    first trials are the oracle's to 1e-9 (test above) and whose value is
    the oracle's objective at the returned parameters."""
    sc = small_ring(C=60, P=3000, huber=True)
    pix = orc.pixels_from_scene(sc)
    out = {}
    for prec in ("f64", "f32"):
        with problem(sc, pix, prec, pcg_maxiter=50, pcg_tol=1e-4, jacobian=jac) as prob:
            costs = _run_until_stall(prob, cap=3000)
            cams, pts = prob.params()
        F_exact = orc.cost(np64(cams), np64(pts), sc.cam_idx, sc.pt_idx, pix, 1.0)
        assert abs(min(costs) - F_exact) <= (1e-12 if prec == "f64" else 1e-6) * F_exact
        out[prec] = min(costs)
    assert abs(out["f32"] - out["f64"]) <= 1e-6 * out["f64"], out


@pytest.mark.parametrize("jac", ["store", "recompute"])
def test_graph_and_direct_launches_are_bitwise_identical(jac):
    sc = small_ring(C=40, P=800, seed=5)
    pix = orc.pixels_from_scene(sc)
    res = []
    for use_graph in (True, False):
        with problem(sc, pix, "f32", pcg_maxiter=30, use_graph=use_graph, jacobian=jac) as prob:
            prob.solve(5)
            st = prob.stats()
            cams, pts = prob.params()
            res.append((st, np64(cams), np64(pts)))
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1]) and np.array_equal(res[0][2], res[1][2])


def test_runs_are_deterministic_and_lm_step_equals_solve():
    sc = small_ring(C=30, P=600, seed=6)
    pix = orc.pixels_from_scene(sc)
    outs = []
    for mode in ("solve", "solve", "step"):
        with problem(sc, pix, "f64", pcg_maxiter=40) as prob:
            if mode == "solve":
                prob.solve(6)
            else:
                for _ in range(6):
                    prob.lm_step()
            outs.append((prob.stats(), np64(prob.params()[0])))
    assert outs[0][0] == outs[1][0] == outs[2][0]
    assert np.array_equal(outs[0][1], outs[1][1]) and np.array_equal(outs[0][1], outs[2][1])


def test_checkpoint_resume_reproduces_trace():
    sc = small_ring(C=30, P=600, seed=8)
    pix = orc.pixels_from_scene(sc)
    with problem(sc, pix, "f64", pcg_maxiter=40) as a:
        a.solve(3)
        state = a.get_state()
        a.solve(4)
        tail_a = a.stats()[-4:]
        pa = np64(a.params()[1])
    with problem(sc, pix, "f64", pcg_maxiter=40) as b:
        b.set_state(state)
        b.solve(4)
        tail_b = b.stats()[-4:]
        pb = np64(b.params()[1])
    assert tail_a == tail_b
    assert np.array_equal(pa, pb)


def test_set_params_and_pixels_reevaluate_cost():
    sc = small_ring(C=20, P=300, seed=9, huber=False)
    pix = orc.pixels_from_scene(sc)
    with problem(sc, pix, "f64") as prob:
        F0, lam0 = prob.scalars()
        assert abs(F0 - orc.cost(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix)) < 1e-10 * F0
        prob.set_params(torch.tensor(sc.cams_gt, device="cuda"), torch.tensor(sc.points_gt, device="cuda"))
        F1, _ = prob.scalars()
        assert abs(F1 - orc.cost(sc.cams_gt, sc.points_gt, sc.cam_idx, sc.pt_idx, pix)) < 1e-10 * F1
        pix2 = pix + 0.5
        prob.set_pixels(torch.tensor(pix2, device="cuda"))
        F2, _ = prob.scalars()
        assert abs(F2 - orc.cost(sc.cams_gt, sc.points_gt, sc.cam_idx, sc.pt_idx, pix2)) < 1e-10 * F2
        prob.solve(3)
        st = prob.stats()
        assert st[0]["cost"] == F2
