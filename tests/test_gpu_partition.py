"""The library's point-partitioned path (ba_set_exchange) on one GPU: the
problem split into two parts, each a Problem driven from its own host
thread, whose exchanges are summed on the host between launches (a
threading barrier: no kernel ever waits for another part's kernel).  The
two parts' common trace equals the unpartitioned library's and the
oracle's, and their points together equal the whole problem's."""
import threading

import numpy as np
import pytest
import torch

import oracle as orc
import paper_2409_12190_gb300 as ba
import scenegen
from gpu_helpers import np64
from paper_2409_12190_gb300.partition import PartProblem, part_arrays, partition_points

pytestmark = pytest.mark.gpu


class HostSum:
    """An in-place sum over n parts, each calling from its own thread."""

    def __init__(self, n):
        self.n = n
        self.bar = threading.Barrier(n, timeout=60)
        self.bufs = [None] * n

    def fn(self, r):
        def allreduce(t):
            torch.cuda.current_stream().synchronize()
            self.bufs[r] = t
            self.bar.wait()
            if r == 0:
                total = self.bufs[0].clone()
                for b in self.bufs[1:]:
                    total += b
                for b in self.bufs:
                    b.copy_(total)
                torch.cuda.synchronize()
            self.bar.wait()
        return allreduce


def _scene(huber):
    return scenegen.ring_scene(40, 1500, seed=11, view_p=1.0 / 7.0, outlier_frac=0.02 if huber else 0.0,
                               outlier_px=20.0, huber_delta=1.0 if huber else 0.0, name="ring-partition")


@pytest.mark.parametrize("prec,huber,nparts", [("f64", True, 2), ("f64", False, 3), ("f32", True, 2)])
def test_parts_reproduce_the_whole_problem(prec, huber, nparts):
    sc = _scene(huber)
    pix = orc.pixels_from_scene(sc)
    iters, maxiter = 6, 15
    opts = ba.Options(precision=prec, pcg_maxiter=maxiter, pcg_tol=1e-4, huber_delta=sc.huber_delta)
    with ba.Problem(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, opts, device="cuda") as whole:
        whole.solve(iters)
        ref = whole.stats()
        cams_w, pts_w = (np64(t) for t in whole.params())
    bounds, _ = partition_points(sc.pt_idx, sc.P, nparts)
    hs = HostSum(nparts)
    parts = []
    for r in range(nparts):
        cams, pts, ci, pi, px, _ = part_arrays(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, bounds, r)
        parts.append(PartProblem(cams, pts, ci, pi, px, hs.fn(r), opts, device="cuda"))
    errors = []

    def run(p):
        try:
            p.solve(iters)
            torch.cuda.synchronize()
        except Exception as e:  # pragma: no cover - reported below
            errors.append(e)

    threads = [threading.Thread(target=run, args=(p,)) for p in parts]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not errors, errors
    traces = [p.stats() for p in parts]
    cams = [np64(p.params()[0]) for p in parts]
    pts = np.concatenate([np64(p.params()[1]) for p in parts])
    for p in parts:
        p.close()
    # every part holds the same trace and cameras
    assert all(t == traces[0] for t in traces)
    assert all(np.array_equal(c, cams[0]) for c in cams)
    tol = 1e-9 if prec == "f64" else 1e-6
    for t, (g, r) in enumerate(zip(traces[0], ref)):
        assert g["accepted"] == r["accepted"] and g["pcg_iters"] == r["pcg_iters"], (t, g, r)
        for key in ("cost", "cost_trial"):
            assert abs(g[key] - r[key]) <= tol * abs(r[key]), (t, key, g[key], r[key])
    if prec == "f64":
        # the parameters too (FP32: only the cost is held, to 1e-6; its
        # parameters differ by FP32 rounding in the two summation orders)
        scale = lambda a: np.maximum(1.0, np.abs(a))  # noqa: E731
        assert np.max(np.abs(cams[0] - cams_w) / scale(cams_w)) < 1e-9
        assert np.max(np.abs(pts - pts_w) / scale(pts_w)) < 1e-9
        # and the oracle's LM
        _, _, oref = orc.lm(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, iters,
                            orc.LMOptions(solver="pcg", pcg_tol=1e-4, pcg_maxiter=maxiter,
                                          huber_delta=sc.huber_delta))
        for g, r in zip(traces[0], oref):
            assert abs(g["cost"] - r["cost"]) <= 1e-9 * abs(r["cost"])


def test_exchange_failure_and_options_are_reported():
    sc = _scene(False)
    pix = orc.pixels_from_scene(sc)

    def bad(t):
        raise RuntimeError("no peer")

    with PartProblem(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, bad,
                     ba.Options(precision="f64", pcg_maxiter=5)) as p:
        with pytest.raises(ba.BAError, match="exchange callback failed"):
            p.solve(1)
    # a partitioned problem uses block-Jacobi PCG
    with pytest.raises(ba.BAError, match="INVALID_ARG"):
        PartProblem(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, lambda t: None,
                    ba.Options(precision="f64", solver="cholesky"))
