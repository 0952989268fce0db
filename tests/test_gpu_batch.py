"""Batched persistent LM (many sliding-window problems in one launch) against
sequential single-problem solves, the FP64 oracle, launch-configuration
invariance (bitwise: the same machine code runs whatever the grid and the
work order), the autotuner and input validation.

The batched kernel runs the single-problem kernels' device code with the
same reduction order, but the compiler forms fused multiply-adds per kernel,
so the two paths agree to rounding, not bit for bit: FP64 per-trial costs to
1e-9 relative, FP32 final costs to the 1e-6 relative bar."""
import numpy as np
import pytest
import torch

import oracle as orc
import paper_2409_12190_gb300 as ba
import scenegen
from gpu_helpers import np64

pytestmark = pytest.mark.gpu

KEYS = ("cost", "cost_trial", "model", "rho", "lam", "pcg_rel_res", "accepted", "pcg_iters",
        "precond_fallbacks")


def _with_heavy_point(seed):
    """A small problem whose point 0 has more observations than one point
    chunk holds (duplicated observations), so the chunk-wide reduction runs."""
    s = scenegen.arc_scene(4, 30, seed=seed, views_lo=2, views_hi=4, name="heavy-point")
    extra = 1100
    ci = np.concatenate([s.cam_idx, (np.arange(extra) % s.C).astype(np.int32)])
    pi = np.concatenate([s.pt_idx, np.zeros(extra, np.int32)])
    rng = np.random.default_rng(seed)
    noise = np.concatenate([s.noise, rng.normal(0.0, 1.0, size=(extra, 2))])
    return scenegen.Scene(cams_gt=s.cams_gt, points_gt=s.points_gt, cam_idx=ci, pt_idx=pi, noise=noise,
                          cams_init=s.cams_init, points_init=s.points_init, name="heavy-point")


def _scenes():
    sc = scenegen.batch_scenes(7, seed=41, p_lo=80.0, p_hi=900.0)
    sc.append(scenegen.arc_scene(1, 60, seed=5, name="one-camera"))
    # each camera sees all 2500 points: two pieces per camera
    sc.append(scenegen.arc_scene(3, 2500, seed=6, views_lo=3, views_hi=3, name="two-pieces"))
    sc.append(scenegen.arc_scene(ba.Batch.MAX_CAMS, 400, seed=7, name="max-cameras"))
    sc.append(_with_heavy_point(8))
    return sc


def _inputs(scenes):
    return [(s.cams_init, s.points_init, s.cam_idx, s.pt_idx, orc.pixels_from_scene(s)) for s in scenes]


def _same_stats(a, b, ctx=""):
    assert len(a) == len(b), ctx
    for t, (x, y) in enumerate(zip(a, b)):
        for k in KEYS:
            vx, vy = x[k], y[k]
            if isinstance(vx, float) and np.isnan(vx):
                assert np.isnan(vy), (ctx, t, k)
            else:
                assert vx == vy, (ctx, t, k, vx, vy)


CONFIGS = [("f32", "auto", 0.0), ("f32", "auto", 1.0), ("f64", "auto", 0.0), ("f64", "recompute", 1.0),
           ("f32", "store", 1.0)]


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.mark.parametrize("prec,jac,huber", CONFIGS)
def test_batch_equals_sequential_single_solves(prec, jac, huber):
    scenes = _scenes()
    inputs = _inputs(scenes)
    # FP64 with a tight PCG keeps both trajectories determined to rounding;
    # FP32 runs both to convergence (Huber's IRLS converges linearly: 250
    # trials, within the batch's 256-record statistics ring) and compares
    # the end
    opts = ba.Options(precision=prec, jacobian=jac, huber_delta=huber, pcg_maxiter=40 if prec == "f32" else 300,
                      pcg_tol=1e-6 if prec == "f32" else 1e-12)
    iters = (250 if huber else 40) if prec == "f32" else 8
    with ba.Batch(inputs, opts) as bt:
        bt.solve(iters)
        bstats = bt.stats(cap=256)
        bparams = bt.params()
        bcost, _ = bt.scalars()
    worst = 0.0
    for b, (s, inp) in enumerate(zip(scenes, inputs)):
        with ba.Problem(*inp, options=opts) as prob:
            prob.solve(iters)
            st = prob.stats()
            cams, pts = prob.params()
            F, _ = prob.scalars()
        assert len(bstats[b]) == len(st) == iters, (s.name, len(bstats[b]), len(st))
        # the starting cost is one fixed-order sum in both paths
        F0 = st[0]["cost"]
        assert bstats[b][0]["cost"] == F0, s.name
        # absolute floors relative to the starting cost for problems whose
        # minimum is (near) zero (one camera: every residual can vanish)
        if prec == "f64":
            for t, (x, y) in enumerate(zip(bstats[b], st)):
                assert abs(x["cost_trial"] - y["cost_trial"]) <= 1e-9 * y["cost"] + 1e-15 * F0, (s.name, t, x, y)
                if abs(y["cost_trial"] - y["cost"]) > 1e-9 * y["cost"] + 1e-15 * F0:
                    assert x["accepted"] == y["accepted"], (s.name, t)
            assert np.max(np.abs(np64(bparams[b][0]) - np64(cams))) <= 1e-7 * max(1.0, float(cams.abs().max()))
            assert np.max(np.abs(np64(bparams[b][1]) - np64(pts))) <= 1e-7 * max(1.0, float(pts.abs().max()))
            allowed = 1e-9 * F + 1e-15 * F0
        elif huber and s.name == "one-camera":
            # one camera: every residual can vanish (a point seen once has
            # three unknowns for two residuals), and under Huber the LM
            # approaches that zero minimum only slowly (250 trials remove
            # ~90 % of the cost, still ~0.2 % per 10 trials), so neither run
            # has converged.  Nor is one trial comparable: the points absorb
            # the camera, so S = U* - sum W V*^-1 W^T cancels down to the
            # damping term and FP32 keeps no digit of it (the two summation
            # orders gave first trials 17 % and 3x apart).  What holds at
            # any precision: LM accepts only decreases, so both runs' costs
            # fall monotonically, and both end far below the start
            for run in (bstats[b], st):
                costs = [t["cost"] for t in run]
                assert all(c1 <= c0 for c0, c1 in zip(costs, costs[1:])) and costs[-1] < 0.2 * F0, s.name
            continue
        else:
            # FP32, both converged: the 1e-6 bar, with an absolute floor of
            # 1e-7 of the starting cost for a problem whose minimum is zero
            # (one camera, plain loss: every residual can vanish, and the
            # two runs reach FP32's noise floor by different paths)
            assert st[-10]["cost"] - F <= 1e-6 * F + 1e-7 * F0, (s.name, "single run not converged")
            allowed = 1e-6 * F + 1e-7 * F0
        worst = max(worst, _rel(bcost[b], F))
        assert abs(bcost[b] - F) <= allowed, (s.name, bcost[b], F, allowed)
        assert bcost[b] < F0, s.name
    print(f"largest relative final-cost difference {worst:.2e}")


def test_batch_split_solves_equal_one_solve():
    inputs = _inputs(_scenes()[:6])
    opts = ba.Options(precision="f32", huber_delta=1.0, pcg_maxiter=30, pcg_tol=1e-5)
    with ba.Batch(inputs, opts) as one, ba.Batch(inputs, opts) as two:
        one.solve(6)
        two.solve(2)
        two.solve(4)
        for b in range(one.n):
            _same_stats(one.stats()[b], two.stats()[b], ctx=b)
        for (c1, p1), (c2, p2) in zip(one.params(), two.params()):
            assert torch.equal(c1, c2) and torch.equal(p1, p2)


@pytest.mark.parametrize("variant", [0, 1])
def test_batch_launch_configuration_does_not_change_results(variant):
    inputs = _inputs(scenegen.batch_scenes(24, seed=43, p_lo=100.0, p_hi=1500.0))
    opts = ba.Options(precision="f32", pcg_maxiter=25, pcg_tol=1e-5)
    with ba.Batch(inputs, opts) as bt:
        ref = None
        for ctas, order in [(1, 0), (2, 1), (3, 0), (1, 1)]:
            bt.reset()
            bt.set_launch(ctas, variant, order)
            assert bt.launch()["grid"] == min(bt.n, ctas * torch.cuda.get_device_properties(0).multi_processor_count)
            bt.solve(4)
            got = (bt.stats(), bt.params(split=False))
            if ref is None:
                ref = got
                continue
            for b in range(bt.n):
                _same_stats(ref[0][b], got[0][b], ctx=(ctas, order, b))
            assert torch.equal(ref[1][0], got[1][0]) and torch.equal(ref[1][1], got[1][1])


def test_batch_f64_matches_oracle_per_trial():
    scenes = scenegen.batch_scenes(4, seed=44, p_lo=60.0, p_hi=200.0)
    inputs = _inputs(scenes)
    iters = 8
    opts = ba.Options(precision="f64", pcg_maxiter=9 * 20 * 3, pcg_tol=1e-14)
    with ba.Batch(inputs, opts) as bt:
        bt.solve(iters)
        bstats = bt.stats(cap=256)
        bparams = bt.params()
    for b, (s, inp) in enumerate(zip(scenes, inputs)):
        c_ref, p_ref, ref = orc.lm(s.cams_init, s.points_init, s.cam_idx, s.pt_idx, inp[4], iters,
                                   orc.LMOptions(solver="cholesky"))
        for g, r in zip(bstats[b], ref):
            assert abs(g["cost_trial"] - r["cost_trial"]) <= 1e-9 * r["cost"], (b, g, r)
            # a trial that changes the cost by less than that tolerance is
            # decided by rounding: its accept flag is compared only above it
            if abs(r["cost_trial"] - r["cost"]) > 1e-9 * r["cost"]:
                assert g["accepted"] == r["accepted"]
        scale = max(np.max(np.abs(c_ref)), 1.0)
        assert np.max(np.abs(np64(bparams[b][0]) - c_ref)) <= 1e-7 * scale
        assert np.max(np.abs(np64(bparams[b][1]) - p_ref)) <= 1e-7 * max(np.max(np.abs(p_ref)), 1.0)


def test_batch_reset_restarts_from_given_parameters():
    scenes = scenegen.batch_scenes(5, seed=45, p_lo=100.0, p_hi=400.0)
    inputs = _inputs(scenes)
    opts = ba.Options(precision="f32", pcg_maxiter=20)
    with ba.Batch(inputs, opts) as bt:
        bt.solve(3)
        first = bt.stats()
        bt.solve(2)
        bt.reset()
        bt.solve(3)
        again = bt.stats()
        for b in range(bt.n):
            _same_stats(first[b], again[b], ctx=b)
        # explicit parameters (the ground truth): the cost starts at the noise floor
        cams = np.concatenate([s.cams_gt for s in scenes])
        pts = np.concatenate([s.points_gt for s in scenes])
        bt.reset(torch.from_numpy(cams), torch.from_numpy(pts))
        bt.solve(1)
        for b, s in enumerate(scenes):
            F0 = 0.5 * float(np.sum(s.noise ** 2))
            assert abs(bt.stats()[b][0]["cost"] - F0) <= 1e-3 * F0


def test_batch_autotune_keeps_results_and_caches(tmp_path):
    inputs = _inputs(scenegen.batch_scenes(40, seed=46, p_lo=100.0, p_hi=1200.0))
    opts = ba.Options(precision="f32", pcg_maxiter=20)
    cache = tmp_path / "tune.jsonl"
    with ba.Batch(inputs, opts) as bt:
        bt.solve(3)
        ref_stats, ref_params = bt.stats(), bt.params(split=False)
        ref_cost = np.asarray(bt.scalars()[0])
        bt.reset()
        cfg, ms = bt.autotune(3, cache)
        assert ms > 0.0 and cache.exists()
        assert {"piece_max", "chunk_slots", "chunk_pts", "ctas_per_sm", "variant", "order"} <= set(cfg)
        # the tuner restored the batch's state
        assert all(len(s) == 0 for s in bt.stats())
        bt.solve(3)
        # the chosen segments pass the tuner's gate: every final cost within
        # 1e-6 of the default cut's
        cost = np.asarray(bt.scalars()[0])
        assert np.all(np.abs(cost - ref_cost) <= 1e-6 * np.abs(ref_cost))
        # the launch configuration alone never changes a result: at the
        # default segments the tuned launch reproduces the first run bit for bit
        bt.set_segments()
        bt.reset()
        bt.solve(3)
        for b in range(bt.n):
            _same_stats(ref_stats[b], bt.stats()[b], ctx=b)
        got = bt.params(split=False)
        assert torch.equal(ref_params[0], got[0]) and torch.equal(ref_params[1], got[1])
    with ba.Batch(inputs, opts) as bt2:
        cfg2, ms2 = bt2.autotune(3, cache)
        assert ms2 == 0.0 and cfg2 == cfg


@pytest.mark.parametrize("seg", [(256, 256, 128), (512, 512, 256), (1024, 1024, 512), (32, 32, 8)])
def test_batch_segments_change_only_rounding(seg):
    """Another cut of the pieces and point chunks reorders some sums only:
    FP64 with a tight PCG follows the oracle's LM trial by trial at 1e-9 on
    sampled problems (the heavy point, wider than a 32-slot chunk, takes the
    block-reduced path), and the FP32 final costs of converged runs stay
    within 1e-6 of the default cut's."""
    scenes = _scenes()
    inputs = _inputs(scenes)
    opts = ba.Options(precision="f64", pcg_maxiter=300, pcg_tol=1e-12)
    with ba.Batch(inputs, opts) as bt:
        bt.set_segments(*seg)
        assert bt.segments() == dict(piece_max=seg[0], chunk_slots=seg[1], chunk_pts=seg[2])
        bt.solve(6)
        bst = bt.stats()
    for b in (0, 3, len(scenes) - 2, len(scenes) - 1):
        s = scenes[b]
        _, _, ref = orc.lm(s.cams_init, s.points_init, s.cam_idx, s.pt_idx, inputs[b][4], 6,
                           orc.LMOptions(solver="cholesky", huber_delta=0.0))
        F0 = ref[0]["cost"]
        for t, (x, y) in enumerate(zip(bst[b], ref)):
            assert abs(x["cost"] - y["cost"]) <= 1e-9 * y["cost"] + 1e-15 * F0, (s.name, t, x, y)
    o32 = ba.Options(precision="f32", pcg_maxiter=40, pcg_tol=1e-6)
    with ba.Batch(inputs, o32) as d, ba.Batch(inputs, o32) as c:
        c.set_segments(*seg)
        d.solve(40)
        c.solve(40)
        Fd = np.asarray(d.scalars()[0])
        Fc = np.asarray(c.scalars()[0])
    # an absolute floor of 1e-7 of the noise energy for the one-camera
    # problem, whose minimum is zero
    ok = np.abs(Fc - Fd) <= 1e-6 * Fd + 1e-7 * np.array([0.5 * float(np.sum(s.noise ** 2)) for s in scenes])
    assert np.all(ok), (Fc, Fd)


def test_batch_rejects_bad_inputs():
    s = scenegen.arc_scene(5, 40, seed=9)
    good = (s.cams_init, s.points_init, s.cam_idx, s.pt_idx, orc.pixels_from_scene(s))
    # a point nobody observes
    pts = np.concatenate([s.points_init, np.zeros((1, 3))])
    with pytest.raises(ba.BAError, match="INVALID_ARG"):
        ba.Batch([good, (s.cams_init, pts, s.cam_idx, s.pt_idx, good[4])])
    # a local camera index out of range
    ci = s.cam_idx.copy()
    ci[3] = s.C
    with pytest.raises(ba.BAError, match="INVALID_ARG"):
        ba.Batch([good, (s.cams_init, s.points_init, ci, s.pt_idx, good[4])])
    # too many cameras
    big = scenegen.arc_scene(ba.Batch.MAX_CAMS + 1, 40, seed=10)
    with pytest.raises(ba.BAError, match="INVALID_ARG"):
        ba.Batch([(big.cams_init, big.points_init, big.cam_idx, big.pt_idx, orc.pixels_from_scene(big))])
