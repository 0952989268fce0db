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


def test_ring_f64_truncated_pcg_within_oracle_order_band():
    """With 50 PCG iterations the reduced system of the ring scene is so
    ill-conditioned that two FP64 CG runs differing only in summation order
    drift apart (the oracle against itself with the observations permuted).
    The GPU trace must stay inside 10x that band of the oracle trace, and
    every accept decision whose margin is outside 10x the band of the trial
    cost must match (on this scene, all but the last: the oracle rejects
    trial 4 by 29 while its permuted run moves that trial cost by 6)."""
    sc = small_ring()
    pix = orc.pixels_from_scene(sc)
    iters = 4
    opts = orc.LMOptions(solver="pcg", pcg_tol=1e-4, pcg_maxiter=50, huber_delta=1.0)
    _, _, ref = orc.lm(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, iters, opts)
    perm = np.random.default_rng(0).permutation(sc.O)
    _, _, ref2 = orc.lm(sc.cams_init, sc.points_init, sc.cam_idx[perm], sc.pt_idx[perm], pix[perm],
                        iters, opts)
    # costs of the accepted states (rejected trial points are dominated by the
    # noise of the unconverged directions and are not compared)
    band = max(_trace_rel(ref2, ref, "cost"), 1e-9)
    with problem(sc, pix, "f64", pcg_maxiter=50, pcg_tol=1e-4) as prob:
        prob.solve(iters)
        gpu = prob.stats()
    # an accept decision is the method's only where the oracle's margin
    # |F' - F| exceeds 10x the drift of its own trial cost under a
    # permutation of the observations (the band criterion applied to F')
    for t, (g, r, r2) in enumerate(zip(gpu, ref, ref2)):
        if abs(r["cost_trial"] - r["cost"]) > 10 * abs(r2["cost_trial"] - r["cost_trial"]):
            assert g["accepted"] == r["accepted"], (t, g, r)
    assert sum(1 for g, r in zip(gpu, ref) if g["accepted"] == r["accepted"]) >= iters - 1
    assert _trace_rel(gpu, ref, "cost") < 10 * band


def _converged_cost(trace):
    acc = [t["cost_trial"] for t in trace if t["accepted"]]
    return min([trace[0]["cost"]] + acc)


@pytest.mark.parametrize("jac", ["store", "recompute"])
@pytest.mark.parametrize("huber", [True, False])
def test_ring_f32_reaches_fp64_final_cost(huber, jac):
    """FP32 per-observation arithmetic reaches the FP64 final cost within 1e-6.

    Plain loss: after 25 trials both runs have converged (quadratic rate).
    Huber: IRLS without the rho'' term converges linearly -- on the outlier
    residuals the true loss is linear, so the gain ratio tends to 2 and each
    trial removes only a small fraction of the remaining excess -- and after
    25 trials the FP64 run still drops ~5e-7 per trial.  There the FP32 cost
    must be within 1e-6 of the FP64 cost plus the decrease of the FP64 run
    over its last three trials (the FP32 run may lag by a rejected trial)."""
    sc = small_ring(C=60, P=3000, huber=huber)
    pix = orc.pixels_from_scene(sc)
    iters = 25
    delta = 1.0 if huber else 0.0
    opts = orc.LMOptions(solver="pcg", pcg_tol=1e-4, pcg_maxiter=50, huber_delta=delta)
    _, _, ref = orc.lm(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, iters, opts)
    F_ref = _converged_cost(ref)
    tail = (ref[-3]["cost"] - F_ref) if huber else 0.0
    with problem(sc, pix, "f32", pcg_maxiter=50, pcg_tol=1e-4, jacobian=jac) as prob:
        prob.solve(iters)
        gpu = prob.stats()
        cams, pts = prob.params()
    F32 = _converged_cost(gpu)
    # re-evaluate the FP32 result in FP64 with the oracle's cost
    F32_exact = orc.cost(np64(cams), np64(pts), sc.cam_idx, sc.pt_idx, pix, delta)
    assert abs(F32_exact - F_ref) < 1e-6 * F_ref + tail
    assert abs(F32 - F_ref) < 1e-6 * F_ref + tail


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
