"""Pose-graph optimisation (the paper's Sec. IV-D, Eqs. 3-4) on the GPU: a
thin binding over the ``ba_pgo_*`` entry points of include/ba.h (argument
marshalling only; every step runs in the library's kernels).

    g = PoseGraph(poses, ei, ej, meas, info, fixed=[0])
    g.solve(20)
    poses = g.poses()

Poses are [N, 7] (tx, ty, tz, qx, qy, qz, qw); meas [E, 7] the measured
relative poses T_e of the edges (ei[e], ej[e]); info [E, 21] the upper
triangles of the edges' 6 x 6 information matrices, row by row.  The cost is
1/2 sum_e r_e^T Omega_e r_e with r_e = Log(zeta_i^-1 zeta_j T_e^-1).
"""
from __future__ import annotations

import ctypes as ct

import torch

from . import _lib
from . import Options, _L, _dev, _ptr, _stats_dict, _stream


class PoseGraph:
    """One pose graph resident on the GPU (FP64).  ``fixed``: indices of the
    poses held in place (default: pose 0, which fixes the gauge), or a
    boolean mask [N], or an empty list for none."""

    def __init__(self, poses, ei, ej, meas, info, fixed=(0,), options: Options | None = None, device="cuda",
                 stream=None):
        self.options = options or Options()
        if self.options.precision != "f64":
            raise ValueError("pose graphs run in FP64")
        self.device = torch.device(device)
        poses = _dev(poses, torch.float64, self.device)
        ei = _dev(ei, torch.int32, self.device)
        ej = _dev(ej, torch.int32, self.device)
        meas = _dev(meas, torch.float64, self.device)
        info = _dev(info, torch.float64, self.device)
        N, E = int(poses.shape[0]), int(ei.shape[0])
        if tuple(poses.shape) != (N, 7) or tuple(ej.shape) != (E,) or tuple(meas.shape) != (E, 7) \
                or tuple(info.shape) != (E, 21) or ei.dim() != 1:
            raise ValueError("poses [N, 7], ei / ej [E], meas [E, 7] and info [E, 21] expected "
                             f"(got {tuple(poses.shape)}, {tuple(ei.shape)}, {tuple(ej.shape)}, "
                             f"{tuple(meas.shape)}, {tuple(info.shape)})")
        mask = None
        if fixed is not None:
            f = torch.as_tensor(fixed)
            if f.dtype == torch.bool:
                if tuple(f.shape) != (N,):
                    raise ValueError("a fixed mask must be [N]")
                mask = f.to(torch.uint8)
            elif f.numel() > 0:
                if int(f.min()) < 0 or int(f.max()) >= N:
                    raise ValueError("fixed pose index out of range")
                mask = torch.zeros(N, dtype=torch.uint8)
                mask[f.long()] = 1
            if mask is not None:
                mask = mask.to(self.device).contiguous()
        self.N, self.E = N, E
        h = ct.c_void_p()
        o = self.options.to_c()
        _lib.check(_L().ba_pgo_create(ct.byref(h), N, E, _ptr(poses), _ptr(ei), _ptr(ej), _ptr(meas), _ptr(info),
                                      _ptr(mask), ct.byref(o), _stream(stream)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _L().ba_pgo_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def solve(self, iters: int, stream=None):
        _lib.check(_L().ba_pgo_solve(self._h, int(iters), _stream(stream)))

    def poses(self, stream=None):
        out = torch.empty(self.N, 7, dtype=torch.float64, device=self.device)
        _lib.check(_L().ba_pgo_get_poses(self._h, _ptr(out), _stream(stream)))
        return out

    def set_poses(self, poses, stream=None):
        p = _dev(poses, torch.float64, self.device)
        if tuple(p.shape) != (self.N, 7):
            raise ValueError("poses must be [N, 7]")
        _lib.check(_L().ba_pgo_set_poses(self._h, _ptr(p), _stream(stream)))

    def stats(self, cap: int = 4096):
        buf = (_lib.ba_iter_stats * cap)()
        n = ct.c_int()
        _lib.check(_L().ba_pgo_get_stats(self._h, buf, cap, ct.byref(n)))
        return [_stats_dict(buf[k]) for k in range(n.value)]

    def scalars(self):
        F, lam = ct.c_double(), ct.c_double()
        _lib.check(_L().ba_pgo_get_scalars(self._h, ct.byref(F), ct.byref(lam)))
        return F.value, lam.value

    def set_lambda(self, lam: float):
        _lib.check(_L().ba_pgo_set_lambda(self._h, float(lam)))

    def linearize(self, stream=None):
        """dict of r [E,6], A [E,6,6], B [E,6,6], Hd [N,21], g [N,6], cost."""
        f = dict(dtype=torch.float64, device=self.device)
        r, A, B = torch.empty(self.E, 6, **f), torch.empty(self.E, 6, 6, **f), torch.empty(self.E, 6, 6, **f)
        Hd, g = torch.empty(self.N, 21, **f), torch.empty(self.N, 6, **f)
        F = ct.c_double()
        _lib.check(_L().ba_pgo_linearize(self._h, _ptr(r), _ptr(A), _ptr(B), _ptr(Hd), _ptr(g), ct.byref(F),
                                         _stream(stream)))
        return dict(r=r, A=A, B=B, Hd=Hd, g=g, cost=F.value)

    def matvec(self, lam: float, x, stream=None):
        x = _dev(x, torch.float64, self.device)
        if tuple(x.shape) != (self.N, 6):
            raise ValueError("x must be [N, 6]")
        y = torch.empty_like(x)
        _lib.check(_L().ba_pgo_matvec(self._h, float(lam), _ptr(x), _ptr(y), _stream(stream)))
        return y

    def damped_solve(self, lam: float, maxiter: int, tol: float, stream=None):
        dx = torch.empty(self.N, 6, dtype=torch.float64, device=self.device)
        its, rel = ct.c_int(), ct.c_double()
        _lib.check(_L().ba_pgo_damped_solve(self._h, float(lam), int(maxiter), float(tol), _ptr(dx),
                                            ct.byref(its), ct.byref(rel), _stream(stream)))
        return dx, its.value, rel.value


def synthesize(poses_gt, ei, ej, noise, drift=None, device="cuda", stream=None):
    """The measurements Exp(noise_e) zeta_i^-1 zeta_j [E, 7] and, with drift,
    the initial estimate Exp(drift_n) zeta_n [N, 7] of a synthetic graph."""
    dev = torch.device(device)
    g = _dev(poses_gt, torch.float64, dev)
    i32 = [_dev(t, torch.int32, dev) for t in (ei, ej)]
    nz = _dev(noise, torch.float64, dev)
    N, E = int(g.shape[0]), int(i32[0].shape[0])
    if tuple(g.shape) != (N, 7) or tuple(i32[1].shape) != (E,) or tuple(nz.shape) != (E, 6):
        raise ValueError("poses_gt [N, 7], ei / ej [E], noise [E, 6] expected")
    meas = torch.empty(E, 7, dtype=torch.float64, device=dev)
    init = None
    dr = None
    if drift is not None:
        dr = _dev(drift, torch.float64, dev)
        if tuple(dr.shape) != (N, 6):
            raise ValueError("drift must be [N, 6]")
        init = torch.empty(N, 7, dtype=torch.float64, device=dev)
    _lib.check(_L().ba_pgo_synthesize(N, E, _ptr(g), _ptr(i32[0]), _ptr(i32[1]), _ptr(nz), _ptr(dr), _ptr(meas),
                                      _ptr(init), _stream(stream)))
    return meas, init
