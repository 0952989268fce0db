"""The direct solver of the reduced camera system (the paper's Cholesky
variant, Sec. IV-C): S formed explicitly on the GPU, a tiled FP64
Cholesky factorisation and triangular solves, against the oracle's explicit
Schur complement and dense Cholesky (oracle.solve_damped with
solver="cholesky"), which its pins tie to the dense solve of Eq. 2."""
import numpy as np
import pytest
import torch

import oracle as orc
import scenegen
from gpu_helpers import np64, problem, rel_err, small_ring

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("jac", ["store", "recompute"])
def test_ba16_f64_cholesky_trace_matches_oracle(jac):
    sc = scenegen.config_scene("ba16")
    pix = orc.pixels_from_scene(sc)
    iters = 20
    cams_ref, pts_ref, ref = orc.lm(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, iters,
                                    orc.LMOptions(solver="cholesky"))
    with problem(sc, pix, "f64", solver="cholesky", jacobian=jac) as prob:
        prob.solve(iters)
        gpu = prob.stats()
        cams, pts = prob.params()
    assert len(gpu) == iters
    for t, (g, r) in enumerate(zip(gpu, ref)):
        for key in ("cost", "cost_trial"):
            assert abs(g[key] - r[key]) <= 1e-9 * abs(r[key]), (t, key, g[key], r[key])
        assert g["pcg_iters"] == 0 and g["precond_fallbacks"] == 0
    assert np.max(np.abs(np64(cams) - cams_ref) / np.maximum(1.0, np.abs(cams_ref))) < 1e-7
    assert np.max(np.abs(np64(pts) - pts_ref) / np.maximum(1.0, np.abs(pts_ref))) < 1e-7


@pytest.mark.parametrize("gauge", [False, True])
def test_damped_solve_cholesky_matches_oracle(gauge):
    """One damped solve on a Huber ring of 250 cameras (n = 2,250 unknowns,
    71 blocks of the factorisation: every kernel's ragged last block), with
    and without the gauge frozen (rows and columns of frozen parameters
    replaced by the identity)."""
    sc = small_ring()
    pix = orc.pixels_from_scene(sc)
    lam = 1e-3
    fixed = orc.gauge_mask(sc.C) if gauge else None
    blk = orc.assemble(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, sc.huber_delta)
    dc_ref, dp_ref, _, _ = orc.solve_damped(blk, sc.cam_idx, sc.pt_idx, lam,
                                            orc.LMOptions(solver="cholesky"), fixed=fixed)
    with problem(sc, pix, "f64", solver="cholesky") as prob:
        if gauge:
            prob.set_fixed(torch.from_numpy(fixed))
        dc, dp, its, rel = prob.damped_solve(lam, 0, 0.0)
    assert its == 0 and rel == 0.0
    assert rel_err(np64(dc), dc_ref) < 1e-9
    assert rel_err(np64(dp), dp_ref) < 1e-9
    if gauge:
        assert np.all(np64(dc)[fixed] == 0.0)


def test_f32_cholesky_reaches_the_oracles_converged_cost():
    """FP32 per-observation arithmetic with the FP64 direct solve: the final
    cost, re-evaluated by the oracle at the returned parameters, is within
    1e-6 of the oracle's converged cost (plain loss, exact solves: converged
    in a few trials)."""
    sc = small_ring(C=60, P=3000, huber=False)
    pix = orc.pixels_from_scene(sc)
    iters = 15
    _, _, ref = orc.lm(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, iters,
                       orc.LMOptions(solver="cholesky"))
    F_ref = min([ref[0]["cost"]] + [t["cost_trial"] for t in ref if t["accepted"]])
    assert ref[-5]["cost"] - F_ref <= 1e-12 * F_ref
    with problem(sc, pix, "f32", solver="cholesky") as prob:
        prob.solve(iters)
        cams, pts = prob.params()
        F32, _ = prob.scalars()
    F_exact = orc.cost(np64(cams), np64(pts), sc.cam_idx, sc.pt_idx, pix)
    assert abs(F_exact - F_ref) <= 1e-6 * F_ref
    # the FP32 variant's cost is the FP64 objective at its (FP32) parameters
    # and its (FP32-rounded) pixels
    pix32 = pix.astype(np.float32).astype(np.float64)
    F_exact32 = orc.cost(np64(cams), np64(pts), sc.cam_idx, sc.pt_idx, pix32)
    assert abs(F32 - F_exact32) <= 1e-12 * F_exact32


def test_cholesky_option_limits():
    import paper_2409_12190_gb300 as ba
    sc = scenegen.arc_scene(6, 60, seed=3, views_lo=3, views_hi=5)
    pix = orc.pixels_from_scene(sc)
    with pytest.raises(ValueError):
        ba.Options(solver="lu").to_c()
    # the dense matrix is limited to 9C <= BA_DENSE_MAX_DIM unknowns
    C = 18432 // 9 + 1
    cams = np.tile(sc.cams_init[:1], (C, 1))
    with pytest.raises(ba.BAError, match="INVALID_ARG"):
        ba.Problem(cams, sc.points_init, np.zeros(sc.O, np.int32) + (C - 1), sc.pt_idx, pix,
                   ba.Options(solver="cholesky"), device="cuda")
