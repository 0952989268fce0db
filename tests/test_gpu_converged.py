"""Parity of the workload configurations at full size, at the tolerances the
method is held to: FP64 per-trial cost within 1e-9 relative and final
parameters within 1e-7; FP32 final cost within 1e-6 relative of the
converged FP64 cost.  No allowance for unconverged tails: every FP32 gate
runs both sides to convergence.

* ba250 (250 cameras, 60,000 points, 480k observations, Huber), FP64, with
  the reduced camera system solved to convergence (GPU: block-Jacobi PCG to
  1e-12 relative residual; oracle: explicit Schur complement and a dense
  Cholesky factorisation, the paper's direct solver of Sec. IV-C).  With
  exact solves the LM trajectory is unique: the oracle against itself with
  the observations permuted moves costs by ~1e-16 and parameters by ~1e-11,
  so the 1e-9 / 1e-7 bar is well posed.  (With PCG truncated at 50
  iterations the oracle's own trajectory moves by ~1e-9 in cost and ~5e-4
  in parameters under the same permutation: no implementation can be held
  to 1e-9 there beyond the first trials, which test_gpu_fullsize checks.)
* ba250, FP32 against FP64, both in the workload's settings (Huber, PCG
  maxiter 50, tol 1e-4), each run until its cost stops decreasing or for
  2,000 trials: the FP32 variant reaches the FP64 cost.
* ba4000 (4,000 cameras, 1.2M points, 8.04M observations), FP32 in the
  benchmark's configuration, run until it stalls, against F_ref: the
  converged FP64 cost (FP64 trials with a tight PCG from the FP32 result
  until an accepted trial gains less than 1e-9).  F_ref is checked against
  the oracle: its objective at the returned parameters, and the gradient
  rows of sampled cameras (computed by the oracle on their sub-problem),
  which must have collapsed from their values at the start.
"""
import os
import sys

import numpy as np
import pytest
import torch

import oracle as orc
import paper_2409_12190_gb300 as ba
import scenegen
from fullsize_helpers import camera_closure, chunked_cost
from gpu_helpers import np64, oracle_pixels_chunked, problem

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402  (the benchmark's F_ref rule, reused as is)


def _costs(trace):
    return [t["cost_trial"] if t["accepted"] else t["cost"] for t in trace]


def _run_until_stall(prob, cap, window=50, rel=1e-10):
    """LM trials in windows until a window lowers the cost by less than rel
    (relative) or cap trials ran; returns the per-trial costs."""
    costs = []
    while len(costs) < cap:
        prob.solve(window)
        costs += _costs(prob.stats(cap=window))
        if len(costs) > window and costs[-window - 1] - costs[-1] <= rel * costs[-1]:
            break
    return costs


@pytest.fixture(scope="module")
def ba250():
    sc = scenegen.config_scene("ba250")
    return sc, orc.pixels_from_scene(sc)


@pytest.fixture(scope="module")
def ba250_exact_ref(ba250):
    """The oracle's LM with exact solves (explicit Schur, dense Cholesky)."""
    sc, pix = ba250
    iters = 8
    return orc.lm(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, iters,
                  orc.LMOptions(solver="cholesky", huber_delta=1.0))


@pytest.mark.parametrize("solver", ["pcg", "cholesky"])
def test_ba250_f64_solved_trials_match_oracle_cholesky(ba250, ba250_exact_ref, solver):
    """FP64 with the reduced system solved to convergence, by the GPU's PCG
    (tolerance 1e-12) or by its direct solver (explicit S, blocked
    Cholesky), against the oracle's explicit Schur complement and dense
    Cholesky: per-trial cost 1e-9, final parameters 1e-7."""
    sc, pix = ba250
    cams_ref, pts_ref, ref = ba250_exact_ref
    iters = len(ref)
    opts = dict(pcg_maxiter=9 * sc.C, pcg_tol=1e-12) if solver == "pcg" else dict(solver="cholesky")
    with problem(sc, pix, "f64", **opts) as prob:
        prob.solve(iters)
        gpu = prob.stats()
        cams, pts = prob.params()
    assert len(gpu) == iters
    assert [g["accepted"] for g in gpu] == [r["accepted"] for r in ref]
    # the cost of every iterate, and the trial cost of every accepted trial
    # (the next iterate's); a rejected trial's cost is F at a point the
    # method discards (trial 1 here: 11.6M from 4.3M), where the step's
    # residual error meets a large gradient -- only its decision is compared
    for t, (g, r) in enumerate(zip(gpu, ref)):
        assert abs(g["cost"] - r["cost"]) <= 1e-9 * abs(r["cost"]), (t, g["cost"], r["cost"])
        if r["accepted"]:
            assert abs(g["cost_trial"] - r["cost_trial"]) <= 1e-9 * abs(r["cost_trial"]), (t, g, r)
    assert np.max(np.abs(np64(cams) - cams_ref) / np.maximum(1.0, np.abs(cams_ref))) < 1e-7
    assert np.max(np.abs(np64(pts) - pts_ref) / np.maximum(1.0, np.abs(pts_ref))) < 1e-7


def test_ba250_f32_reaches_the_f64_cost(ba250):
    """Huber IRLS without the rho'' term converges only linearly, and on
    ba250 neither precision has stopped decreasing after 2,000 trials (the
    last 50 trials still gain ~1e-7 relative); the two runs follow
    different paths down the same slow valley.  What is well posed is that
    the FP32 variant reaches the FP64 run's final cost: its own final cost,
    an exact FP64 evaluation at its parameters, is at most 1e-6 above it."""
    sc, pix = ba250
    out = {}
    for prec in ("f64", "f32"):
        with problem(sc, pix, prec, pcg_maxiter=50, pcg_tol=1e-4) as prob:
            costs = _run_until_stall(prob, cap=2000)
            F, _ = prob.scalars()
            cams, pts = prob.params()
        # the reported cost is the objective, evaluated in FP64 in both
        # precisions, at the returned parameters and the problem's pixels
        # (FP32-rounded in the FP32 variant)
        px = pix if prec == "f64" else pix.astype(np.float32).astype(np.float64)
        F_exact = orc.cost(np64(cams), np64(pts), sc.cam_idx, sc.pt_idx, px, sc.huber_delta)
        assert abs(F - F_exact) <= 1e-12 * F_exact
        out[prec] = (min(costs), len(costs))
    F64, F32 = out["f64"][0], out["f32"][0]
    print(f"ba250 after {out['f64'][1]} / {out['f32'][1]} trials: FP64 {F64:.10g}, FP32 {F32:.10g} "
          f"({(F32 - F64) / F64:.2e})")
    assert F32 <= (1 + 1e-6) * F64, out


@pytest.fixture(scope="module")
def ba4000():
    sc = scenegen.config_scene("ba4000")
    return sc, oracle_pixels_chunked(sc)


def test_ba4000_f32_converges_to_f_ref(ba4000):
    sc, pix = ba4000
    dev = torch.device("cuda")
    ci = torch.from_numpy(sc.cam_idx).to(dev)
    pi = torch.from_numpy(sc.pt_idx).to(dev)
    px = torch.from_numpy(pix).to(dev)
    # F_ref by the benchmark's rule
    F_ref, info, (cams, pts) = bench.compute_f_ref(sc, ci, pi, px, dev, want_params=True)
    # the FP32 benchmark configuration, run until it stalls
    with bench._problem(sc, ci, pi, px, "f32", dev) as p32:
        costs = _run_until_stall(p32, cap=600)
    F32 = min(costs)
    assert abs(F32 - F_ref) <= 1e-6 * F_ref, (F32, F_ref, info)

    # F_ref against the oracle: the objective at the FP64 parameters, and the
    # gradient rows of sampled cameras, far below their starting values
    cams, pts = np64(cams), np64(pts)
    assert abs(chunked_cost(sc, cams, pts, pix) - F_ref) <= 1e-12 * F_ref
    sel = np.array([0, 1333, 2666, 3999])
    obs, pts_sel, ptl = camera_closure(sc, sel)
    ci_s = sc.cam_idx[obs]
    g_end = orc.assemble(cams, pts[pts_sel], ci_s, ptl, pix[obs])["gc"][sel]
    g_0 = orc.assemble(sc.cams_init, sc.points_init[pts_sel], ci_s, ptl, pix[obs])["gc"][sel]
    ratio = np.linalg.norm(g_end) / np.linalg.norm(g_0)
    print(f"F_ref {F_ref:.10g} ({info['fp64_trials']} FP64 trials, last gain {info['last_accepted_decrease_rel']:.2e}); "
          f"FP32 {F32:.10g} ({(F32 - F_ref) / F_ref:.2e}); gradient rows {ratio:.2e} of their start")
    assert ratio <= 1e-2
