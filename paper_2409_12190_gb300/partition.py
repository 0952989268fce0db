"""Point-partitioned problems: one bundle adjustment split across GPUs.

Each part holds a subset of the points with ALL of their observations and
every camera (replicated).  The library runs the LM trial of each part and,
at its six exchange points (U and gc, the Schur pass's per-camera sums, the
pass-B sums of every PCG iteration, the trial and cost scalars), asks the
caller to sum a device buffer over all parts (``ba_set_exchange``).  This
module partitions the observations, builds the parts and bridges the
exchange to an in-place all-reduce: ``torch.distributed.all_reduce`` with one
GPU per rank, or any function that sums a tensor across the parts.

Not in the paper, which runs on one GPU.  Argument marshalling and host-side
bookkeeping only: every sum and every product runs in the library's kernels.
"""
from __future__ import annotations

import ctypes as ct

import numpy as np
import torch

from . import _lib
from . import Options, Problem

EXCHANGE_FN = _lib.EXCHANGE_FN


def exchange_cap(C: int) -> int:
    """Doubles the exchange buffer must hold (BA_EXCHANGE_CAP)."""
    return 64 * int(C) + 8


def partition_points(pt_idx, P: int, nparts: int):
    """Split points 0..P-1 into nparts contiguous ranges with about equal
    observation counts.  Returns (bounds [nparts + 1] into the point range,
    the part of every observation [O])."""
    pt_idx = np.asarray(pt_idx, dtype=np.int64)
    if nparts < 1:
        raise ValueError("nparts must be >= 1")
    counts = np.bincount(pt_idx, minlength=P)
    cum = np.concatenate([[0], np.cumsum(counts)])
    O = cum[-1]
    bounds = [0]
    for r in range(1, nparts):
        bounds.append(int(np.searchsorted(cum, O * r / nparts, side="left")))
    bounds.append(P)
    bounds = np.maximum.accumulate(np.asarray(bounds, dtype=np.int64))
    part_of_point = np.searchsorted(bounds, np.arange(P), side="right") - 1
    return bounds, part_of_point[pt_idx]


def part_arrays(cams, points, cam_idx, pt_idx, pixels, bounds, r: int):
    """Arrays of part r: every camera, the points in [bounds[r], bounds[r+1])
    renumbered from 0, and their observations in input order.  Returns
    (cams, points, cam_idx, pt_idx, pixels, obs) with obs the observations'
    indices in the whole problem."""
    pt_idx = np.asarray(pt_idx)
    lo, hi = int(bounds[r]), int(bounds[r + 1])
    obs = np.flatnonzero((pt_idx >= lo) & (pt_idx < hi))
    return (np.asarray(cams), np.asarray(points)[lo:hi], np.asarray(cam_idx)[obs].astype(np.int32),
            (pt_idx[obs] - lo).astype(np.int32), np.asarray(pixels)[obs], obs)


class PartProblem:
    """One part of a point-partitioned problem: a ``Problem`` on the part's
    arrays whose exchanges call ``allreduce(t)``, which must sum the 1-D
    device tensor ``t`` over all parts in place (every part calls it in the
    same order).  ``allreduce`` runs with the library's stream current."""

    def __init__(self, cams, points, cam_idx, pt_idx, pixels, allreduce, options: Options | None = None,
                 device="cuda"):
        self.problem = Problem(cams, points, cam_idx, pt_idx, pixels, options, device=device)
        self.device = self.problem.device
        self._allreduce = allreduce
        self.xbuf = torch.zeros(exchange_cap(self.problem.C), dtype=torch.float64, device=self.device)
        self._fn = EXCHANGE_FN(self._exchange)   # kept alive with the object
        _lib.check(_lib.load().ba_set_exchange(self.problem._h, self._fn, None,
                                               ct.c_void_p(self.xbuf.data_ptr()), self.xbuf.numel()))

    def _exchange(self, n, stream, ctx):
        try:
            s = torch.cuda.ExternalStream(stream, device=self.device)
            with torch.cuda.stream(s):
                self._allreduce(self.xbuf[:n])
            return 0
        except Exception:  # reported by the library as a failed trial
            return 1

    def __getattr__(self, name):
        # every other method of the part's Problem (solve, stats, params,
        # set_params, get_state, profile_trials, ...)
        problem = self.__dict__.get("problem")
        if problem is None:
            raise AttributeError(name)
        return getattr(problem, name)

    def close(self):
        if self.problem is not None:
            _lib.load().ba_set_exchange(self.problem._h, EXCHANGE_FN(), None, None, 0)  # NULL: no longer a part
            self.problem.close()
            self.problem = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def dist_allreduce(group=None):
    """An ``allreduce`` for PartProblem over torch.distributed (one part per
    rank; NCCL for device tensors)."""
    import torch.distributed as dist

    def fn(t):
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return fn
