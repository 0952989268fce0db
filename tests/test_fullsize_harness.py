"""The full-size parity tests' harness, checked on the CPU: the oracle's
rows on a camera's point closure equal its rows on the whole problem, and
the LM-rule check accepts the oracle's own traces and catches a changed
decision or damping."""
import copy

import numpy as np
import pytest

import oracle as orc
import paper_2409_12190_gb300 as ba
import scenegen
from fullsize_helpers import DIAG_MAX, DIAG_MIN, camera_closure, damped_U, check_lm_rule, oracle_rows, rand_x


def test_closure_rows_equal_whole_problem_rows():
    sc = scenegen.config_scene("ba250", small=True)
    pix = orc.pixels_from_scene(sc)
    lam = 1e-4
    cams_sel = np.array([0, 17, 125, 249])
    x = rand_x(np.random.default_rng(0), sc.C)
    obs, pts, ptl = camera_closure(sc, cams_sel)
    # every observation of a sampled camera is in the closure, and no point
    # in it misses one of its observations
    assert np.isin(np.flatnonzero(np.isin(sc.cam_idx, cams_sel)), obs).all()
    assert np.array_equal(np.bincount(ptl), np.bincount(sc.pt_idx)[pts])
    assert obs.shape[0] < sc.O
    ref = oracle_rows(sc, pix, cams_sel, lam, x)
    blk = orc.assemble(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, sc.huber_delta)
    Us = damped_U(blk["U"], lam, DIAG_MIN, DIAG_MAX)
    Vinv = orc.point_damped_inverse(blk["V"], lam, DIAG_MIN, DIAG_MAX)
    Sx = orc.schur_matvec(x, Us, Vinv, blk["W"], sc.cam_idx, sc.pt_idx)

    def close(a, b):
        return np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))

    assert close(ref["U"], blk["U"][cams_sel])
    assert close(ref["gc"], blk["gc"][cams_sel])
    assert close(ref["V"], blk["V"][pts])
    assert close(ref["gp"], blk["gp"][pts])
    assert close(ref["Sx"], Sx[cams_sel])


@pytest.fixture(scope="module")
def oracle_trace():
    sc = scenegen.ring_scene(30, 600, seed=3, view_p=1.0 / 5.7)
    pix = orc.pixels_from_scene(sc)
    _, _, tr = orc.lm(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, 8,
                      orc.LMOptions(solver="pcg", pcg_tol=1e-4, pcg_maxiter=50))
    return tr


def test_lm_rule_accepts_the_oracle_trace(oracle_trace):
    assert any(t["accepted"] for t in oracle_trace)
    assert any(not t["accepted"] for t in oracle_trace)
    check_lm_rule(oracle_trace, ba.Options(pcg_maxiter=50))


@pytest.mark.parametrize("plant", ["accepted", "lam", "cost", "rho"])
def test_lm_rule_catches_a_planted_mistake(oracle_trace, plant):
    tr = copy.deepcopy(oracle_trace)
    t = next(i for i, s in enumerate(tr[:-1]) if s["accepted"])
    if plant == "accepted":
        tr[t]["accepted"] = False
    elif plant == "lam":
        tr[t + 1]["lam"] *= 2.0
    elif plant == "cost":
        tr[t + 1]["cost"] = tr[t]["cost"]
    else:
        tr[t]["rho"] = -tr[t]["rho"]
    with pytest.raises(AssertionError):
        check_lm_rule(tr, ba.Options(pcg_maxiter=50))
