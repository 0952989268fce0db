"""The multi-rank path of bench.py (one process per GPU, each rank its own
replica or its own batch of problems, no data-path collective) with two
gloo ranks on the CPU: every rank reports the slowest rank's time, and the
ranks' batches are distinct problems."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, _ = bench.dist_env()
        ms = bench.rank_max(10.0 + 3.0 * r, torch.device("cpu"), w)
        q.put((r, w, ms, bench.batch_seed(r)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_time_by_the_slowest_and_solve_their_own_batches():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, PORT, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == world for o in out)
    # every rank reports the slowest rank's time
    assert all(o[2] == 13.0 for o in out)
    # each rank draws its own batch of problems
    assert out[0][3] != out[1][3]


PORT = _free_port()


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.rank_max(7.5, torch.device("cpu"), 1) == 7.5
    assert bench.batch_seed(0) == 4
