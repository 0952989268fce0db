"""Helpers of the full-size parity tests that need no GPU: the sub-problem
on which the oracle computes sampled rows one by one, a chunked FP64 cost,
and the LM rule every recorded trial must obey (test code only)."""
import numpy as np

import oracle as orc
from oracle.ba_oracle import _ustar as damped_U  # U* = U + lambda clamp(diag U)

# block and product tolerances of the step tests (FP32: a few float ulps of
# the block scale; FP64: association order only)
TOL_BLOCKS = {"f64": 1e-10, "f32": 3e-4}
TOL_MATVEC = {"f64": 1e-10, "f32": 1e-4}
DIAG_MIN, DIAG_MAX = 1e-6, 1e32


def camera_closure(sc, cams_sel):
    """The sub-problem on which the oracle computes sampled rows exactly:
    every observation of every point that one of ``cams_sel`` sees.

    Returns (obs, pts, pt_local): the observation indices (increasing), the
    points (increasing) and the observations' point indices renumbered into
    ``pts``.  U, gc and the Schur-product rows of the sampled cameras, and V,
    gp of every point in ``pts``, are sums over observations all of which the
    sub-problem holds."""
    seen = np.isin(sc.cam_idx, cams_sel)
    pts = np.unique(sc.pt_idx[seen])
    obs = np.flatnonzero(np.isin(sc.pt_idx, pts))
    local = np.full(sc.P, -1, np.int64)
    local[pts] = np.arange(pts.shape[0])
    return obs, pts, local[sc.pt_idx[obs]]


def oracle_rows(sc, pix, cams_sel, lam, x):
    """Oracle blocks and Schur-product rows restricted to ``cams_sel``."""
    obs, pts, ptl = camera_closure(sc, cams_sel)
    ci = sc.cam_idx[obs]
    blk = orc.assemble(sc.cams_init, sc.points_init[pts], ci, ptl, pix[obs], sc.huber_delta)
    Us = damped_U(blk["U"], lam, DIAG_MIN, DIAG_MAX)
    Vinv = orc.point_damped_inverse(blk["V"], lam, DIAG_MIN, DIAG_MAX)
    Sx = orc.schur_matvec(x, Us, Vinv, blk["W"], ci, ptl)
    return dict(U=blk["U"][cams_sel], gc=blk["gc"][cams_sel], V=blk["V"], gp=blk["gp"], pts=pts,
                Sx=Sx[cams_sel])


def chunked_cost(sc, cams, points, pix, chunk=1 << 20):
    return sum(orc.cost(cams, points, sc.cam_idx[a:a + chunk], sc.pt_idx[a:a + chunk],
                        pix[a:a + chunk], sc.huber_delta) for a in range(0, sc.O, chunk))


def rand_x(rng, C):
    """A camera-space vector with the parameters' scales (angles, t, f, k)."""
    return rng.normal(size=(C, 9)) * np.array([1e-3] * 6 + [1.0, 1e-3, 1e-3])


def check_lm_rule(trace, opts):
    """Properties of every trial that hold at any size: the gain ratio is
    (F - F') / Delta L, a trial is accepted iff F' is finite, Delta L > 0 and
    F' < F; theta moves only on acceptance, and lambda follows the
    trust-region rule."""
    for t, s in enumerate(trace):
        assert 0 <= s["pcg_iters"] <= opts.pcg_maxiter, (t, s)
        acc = bool(np.isfinite(s["cost_trial"]) and s["model"] > 0 and s["cost_trial"] < s["cost"])
        assert s["accepted"] == acc, (t, s)
        if s["model"] != 0 and np.isfinite(s["cost_trial"]):
            rho = (s["cost"] - s["cost_trial"]) / s["model"]
            assert abs(s["rho"] - rho) <= 1e-12 * max(1.0, abs(rho)), (t, s)
        if t + 1 < len(trace):
            nxt = trace[t + 1]
            assert nxt["cost"] == (s["cost_trial"] if acc else s["cost"]), t
            if acc and s["rho"] > opts.rho_good:
                lam = max(s["lam"] / opts.up, opts.lambda_min)
            elif not acc or s["rho"] < opts.rho_bad:
                lam = min(s["lam"] / opts.down, opts.lambda_max)
            else:
                lam = s["lam"]
            assert nxt["lam"] == lam, t
