"""The point-partitioned LM on the CPU: two gloo ranks, each holding half of
the points (with all their observations) and every camera, exchange the
six sums of a trial by all-reduce and reproduce the unpartitioned oracle's
LM trace; plus the host-side partitioning of the library's binding."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _scene():
    import scenegen
    return scenegen.ring_scene(40, 1500, seed=11, view_p=1.0 / 7.0, outlier_frac=0.02, outlier_px=20.0,
                               huber_delta=1.0, name="ring-partition")


ITERS = 6
MAXITER = 15


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, HERE)
    import oracle as orc
    from paper_2409_12190_gb300.partition import part_arrays, partition_points
    from partition_oracle import part_lm
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc = _scene()
        pix = orc.pixels_from_scene(sc)
        bounds, _ = partition_points(sc.pt_idx, sc.P, world)
        cams, pts, ci, pi, px, obs = part_arrays(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix,
                                                 bounds, rank)

        def allreduce(a):
            t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
            dist.all_reduce(t)
            return t.numpy()

        opts = orc.LMOptions(solver="pcg", pcg_tol=1e-4, pcg_maxiter=MAXITER, huber_delta=1.0)
        c, p, trace = part_lm(cams, pts, ci, pi, px, ITERS, opts, allreduce)
        q.put((rank, trace, c, p, int(bounds[rank]), len(obs)))
    finally:
        dist.destroy_process_group()


PORT = _free_port()


def test_two_point_partitioned_ranks_reproduce_the_oracle_lm():
    sys.path.insert(0, ROOT)
    import oracle as orc
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, PORT, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in range(world)), key=lambda o: o[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sc = _scene()
    pix = orc.pixels_from_scene(sc)
    opts = orc.LMOptions(solver="pcg", pcg_tol=1e-4, pcg_maxiter=MAXITER, huber_delta=1.0)
    cams_ref, pts_ref, ref = orc.lm(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, ITERS, opts)
    # both parts hold the same (replicated) trace and cameras
    assert out[0][1] == out[1][1]
    assert np.array_equal(out[0][2], out[1][2])
    assert sum(o[5] for o in out) == sc.O
    for t, (g, r) in enumerate(zip(out[0][1], ref)):
        assert g["accepted"] == r["accepted"] and g["pcg_iters"] == r["pcg_iters"], t
        for key in ("cost", "cost_trial", "model"):
            assert abs(g[key] - r[key]) <= 1e-9 * abs(r[key]), (t, key, g[key], r[key])
    assert np.max(np.abs(out[0][2] - cams_ref) / np.maximum(1.0, np.abs(cams_ref))) < 1e-9
    pts = np.concatenate([o[3] for o in out])
    assert np.max(np.abs(pts - pts_ref) / np.maximum(1.0, np.abs(pts_ref))) < 1e-9


def test_partition_points_balances_observations_and_keeps_points_whole():
    sys.path.insert(0, ROOT)
    import scenegen
    from paper_2409_12190_gb300.partition import part_arrays, partition_points
    sc = scenegen.ring_scene(30, 2000, seed=5, view_p=1.0 / 7.0, name="r")
    for n in (1, 2, 3, 8):
        bounds, part = partition_points(sc.pt_idx, sc.P, n)
        assert bounds[0] == 0 and bounds[-1] == sc.P and np.all(np.diff(bounds) >= 0)
        # every observation of a point is in that point's part
        assert np.array_equal(part, np.searchsorted(bounds, sc.pt_idx, side="right") - 1)
        counts = np.bincount(part, minlength=n)
        assert counts.sum() == sc.O
        # balanced to within the largest point's observations
        assert counts.max() - counts.min() <= 2 * np.bincount(sc.pt_idx).max() + sc.O // (10 * n) + 1
        got = 0
        for r in range(n):
            cams, pts, ci, pi, px, obs = part_arrays(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx,
                                                     np.zeros((sc.O, 2)), bounds, r)
            assert cams.shape == sc.cams_init.shape
            assert np.all(pi >= 0) and np.all(pi < pts.shape[0])
            assert np.array_equal(pi + bounds[r], sc.pt_idx[obs])
            got += len(obs)
        assert got == sc.O
    with pytest.raises(ValueError):
        partition_points(sc.pt_idx, sc.P, 0)
