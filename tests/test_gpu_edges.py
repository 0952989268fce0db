"""Edge and degenerate cases: bad indices, non-finite input, a camera with no
observation, points seen once, the smallest problem, no PCG iterations."""
import numpy as np
import pytest
import torch

import oracle as orc
import paper_2409_12190_gb300 as ba
import scenegen
from gpu_helpers import np64, problem

pytestmark = pytest.mark.gpu


def test_index_out_of_range_is_invalid_arg():
    sc = scenegen.arc_scene(4, 30, seed=1)
    pix = orc.pixels_from_scene(sc)
    for field, bad in (("cam_idx", sc.C), ("pt_idx", -1)):
        ci, pi = sc.cam_idx.copy(), sc.pt_idx.copy()
        (ci if field == "cam_idx" else pi)[7] = bad
        with pytest.raises(ba.BAError, match="INVALID_ARG"):
            ba.Problem(sc.cams_init, sc.points_init, ci, pi, pix, ba.Options())


def test_nonfinite_pixel_is_nonfinite():
    sc = scenegen.arc_scene(4, 30, seed=1)
    pix = orc.pixels_from_scene(sc)
    pix[3, 1] = np.nan
    with pytest.raises(ba.BAError, match="NONFINITE"):
        ba.Problem(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, ba.Options())


def test_overflowing_initial_cost_is_nonfinite():
    sc = scenegen.arc_scene(3, 10, seed=2)
    pix = orc.pixels_from_scene(sc)
    cams = sc.cams_init.copy()
    cams[1, 6] = 1e200          # finite focal length, residual^2 overflows
    with pytest.raises(ba.BAError, match="NONFINITE"):
        ba.Problem(cams, sc.points_init, sc.cam_idx, sc.pt_idx, pix, ba.Options())


def test_unobserved_camera_and_single_view_points_match_oracle():
    base = scenegen.arc_scene(5, 60, seed=3, views_lo=1, views_hi=3)
    # add a sixth camera that no observation uses
    cams_init = np.vstack([base.cams_init, base.cams_init[:1]])
    cams_gt = np.vstack([base.cams_gt, base.cams_gt[:1]])
    sc = scenegen.Scene(cams_gt, base.points_gt, base.cam_idx, base.pt_idx, base.noise,
                        cams_init, base.points_init)
    assert np.bincount(sc.pt_idx).min() == 1
    pix = orc.pixels_from_scene(sc)
    iters = 6
    _, _, ref = orc.lm(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, iters,
                       orc.LMOptions(solver="pcg", pcg_maxiter=10, pcg_tol=0.0))
    with problem(sc, pix, "f64", pcg_maxiter=10, pcg_tol=0.0) as prob:
        prob.solve(iters)
        gpu = prob.stats()
        cams, _ = prob.params()
    for g, r in zip(gpu, ref):
        assert abs(g["cost_trial"] - r["cost_trial"]) < 1e-8 * r["cost"]
    # the unobserved camera never moves
    assert np.array_equal(np64(cams)[5], cams_init[5])


def test_single_observation_problem():
    sc = scenegen.arc_scene(1, 1, seed=4, views_lo=1, views_hi=1)
    assert sc.O == 1
    pix = orc.pixels_from_scene(sc)
    _, _, ref = orc.lm(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, 3,
                       orc.LMOptions(solver="pcg", pcg_maxiter=5, pcg_tol=0.0))
    with problem(sc, pix, "f64", pcg_maxiter=5, pcg_tol=0.0) as prob:
        prob.solve(3)
        gpu = prob.stats()
    for g, r in zip(gpu, ref):
        assert abs(g["cost_trial"] - r["cost_trial"]) <= 1e-8 * max(r["cost"], 1e-300) + 1e-20


def test_zero_pcg_iterations_rejects_with_zero_step():
    sc = scenegen.arc_scene(4, 40, seed=5)
    pix = orc.pixels_from_scene(sc)
    with problem(sc, pix, "f64", pcg_maxiter=0) as prob:
        prob.solve(2)
        st = prob.stats()
    # dc = 0, dp = -V*^-1 gp: a point-only step (still a descent direction)
    assert all(s["pcg_iters"] == 0 for s in st)
    _, _, ref = orc.lm(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, 2,
                       orc.LMOptions(solver="pcg", pcg_maxiter=0))
    for g, r in zip(st, ref):
        assert abs(g["cost_trial"] - r["cost_trial"]) < 1e-9 * r["cost"]


def test_zero_residual_problem_stays_at_rounding_level():
    sc = scenegen.arc_scene(3, 20, seed=6, noise_px=0.0, rot_perturb=0.0, t_perturb=0.0,
                            pt_perturb=0.0)
    pix = orc.pixels_from_scene(sc)
    with problem(sc, pix, "f64") as prob:
        prob.solve(3)
        st = prob.stats()
        cams, _ = prob.params()
    assert all(np.isfinite(s["cost_trial"]) and s["cost_trial"] < 1e-18 for s in st)
    assert np.max(np.abs(np64(cams) - sc.cams_gt)) < 1e-9
