"""GB300 (sm_103a) Levenberg-Marquardt bundle adjustment.

A thin Python binding over the C ABI of ``libba_gb300.so`` (include/ba.h):
torch tensors supply device memory and streams, every computation runs in
the library's CUDA kernels.  There is no CPU fallback: without the built
library every call raises.

    import torch, paper_2409_12190_gb300 as ba
    prob = ba.Problem(cams, points, cam_idx, pt_idx, pixels,
                      ba.Options(precision="f32", huber_delta=1.0))
    prob.solve(20)
    cams, points = prob.params()
"""
from __future__ import annotations

import ctypes as ct
import dataclasses

import torch

from . import _lib
from ._lib import BAError, BA_PREC_F32, BA_PREC_F64

__all__ = ["Options", "Problem", "Batch", "project", "csr_build", "kernel_launch_count",
           "BAError", "library_path", "bundle_adjust", "MLP_NPARAM", "MLP_FIN", "mlp_init",
           "mlp_forward", "mlp_loss_grad", "mlp_train", "PoseGraph"]

MLP_NPARAM = _lib.BA_MLP_NPARAM
MLP_FIN = _lib.BA_MLP_FIN
MLP_FOUT = _lib.BA_MLP_FOUT

library_path = _lib.LIB_PATH


def _L():
    return _lib.load()


def _stream(stream=None) -> ct.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ct.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else ct.c_void_p(t.data_ptr())


@dataclasses.dataclass
class Options:
    """Solver options (see ba_options in include/ba.h)."""
    precision: str = "f64"          # "f64" or "f32"
    huber_delta: float = 0.0
    lambda0: float = 1e-4
    up: float = 2.0
    down: float = 0.0625
    rho_good: float = 0.75
    rho_bad: float = 0.25
    lambda_min: float = 1e-16
    lambda_max: float = 1e32
    diag_min: float = 1e-6
    diag_max: float = 1e32
    pcg_maxiter: int = 250
    pcg_tol: float = 1e-4
    use_graph: bool = True
    max_stats: int = 4096
    jacobian: str = "auto"          # "auto", "recompute" or "store"
    solver: str = "pcg"             # "pcg" or "cholesky" (dense direct solve, 9C <= 18432)

    @property
    def dtype(self):
        return torch.float32 if self.precision == "f32" else torch.float64

    def to_c(self) -> _lib.ba_options:
        o = _lib.ba_options()
        _lib.check(_L().ba_options_default(ct.byref(o)))
        if self.precision not in ("f32", "f64"):
            raise ValueError("precision must be 'f32' or 'f64'")
        o.precision = BA_PREC_F32 if self.precision == "f32" else BA_PREC_F64
        for f in ("huber_delta", "lambda0", "up", "down", "rho_good", "rho_bad", "lambda_min",
                  "lambda_max", "diag_min", "diag_max", "pcg_tol"):
            setattr(o, f, float(getattr(self, f)))
        o.pcg_maxiter = int(self.pcg_maxiter)
        o.use_graph = int(bool(self.use_graph))
        o.max_stats = int(self.max_stats)
        if self.jacobian not in _lib.BA_JAC:
            raise ValueError("jacobian must be 'auto', 'recompute' or 'store'")
        o.jacobian_mode = _lib.BA_JAC[self.jacobian]
        if self.solver not in _lib.BA_SOLVER:
            raise ValueError("solver must be 'pcg' or 'cholesky'")
        o.solver = _lib.BA_SOLVER[self.solver]
        return o


def _dev(t, dtype, device):
    t = torch.as_tensor(t)
    return t.to(device=device, dtype=dtype).contiguous()


def _check_problem_shapes(cams, points, cam_idx, pt_idx, pixels):
    """The C ABI takes plain pointers and cannot see buffer sizes: check on
    the host that the arrays agree, so that a wrong shape is an error here
    and never a read past the end of a device buffer."""
    C, P = int(cams.shape[0]), int(points.shape[0])
    O = int(cam_idx.shape[0]) if cam_idx.dim() == 1 else -1
    if tuple(cams.shape) != (C, 9) or tuple(points.shape) != (P, 3):
        raise ValueError(f"cams must be [C, 9] and points [P, 3] (got {tuple(cams.shape)}, {tuple(points.shape)})")
    if O < 0 or tuple(pt_idx.shape) != (O,) or tuple(pixels.shape) != (O, 2):
        raise ValueError(f"cam_idx, pt_idx must be [O] and pixels [O, 2] (got {tuple(cam_idx.shape)}, "
                         f"{tuple(pt_idx.shape)}, {tuple(pixels.shape)})")


class Problem:
    """One bundle-adjustment problem resident on the GPU.

    cams [C, 9] (omega, t, f, k1, k2), points [P, 3], cam_idx / pt_idx [O]
    int32, pixels [O, 2]; any device (copied), float dtype converted to the
    options' precision."""

    def __init__(self, cams, points, cam_idx, pt_idx, pixels, options: Options | None = None,
                 device="cuda", stream=None):
        self.options = options or Options()
        self.dtype = self.options.dtype
        self.device = torch.device(device)
        _check_problem_shapes(*(torch.as_tensor(t) for t in (cams, points, cam_idx, pt_idx, pixels)))
        cams = _dev(cams, self.dtype, self.device)
        points = _dev(points, self.dtype, self.device)
        ci = _dev(cam_idx, torch.int32, self.device)
        pi = _dev(pt_idx, torch.int32, self.device)
        px = _dev(pixels, self.dtype, self.device)
        self.C, self.P, self.O = int(cams.shape[0]), int(points.shape[0]), int(ci.shape[0])
        h = ct.c_void_p()
        o = self.options.to_c()
        _lib.check(_L().ba_problem_create(ct.byref(h), self.C, self.P, self.O, _ptr(cams),
                                          _ptr(points), _ptr(ci), _ptr(pi), _ptr(px), ct.byref(o),
                                          _stream(stream)))
        self._h = h

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            _L().ba_problem_destroy(self._h)
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

    # -- LM -----------------------------------------------------------------
    def lm_step(self, stream=None):
        _lib.check(_L().ba_lm_step(self._h, _stream(stream)))

    def solve(self, iters: int, stream=None):
        _lib.check(_L().ba_solve(self._h, int(iters), _stream(stream)))

    def params(self, stream=None):
        cams = torch.empty((self.C, 9), dtype=self.dtype, device=self.device)
        pts = torch.empty((self.P, 3), dtype=self.dtype, device=self.device)
        _lib.check(_L().ba_get_params(self._h, _ptr(cams), _ptr(pts), _stream(stream)))
        return cams, pts

    def _check(self, t, shape, what):
        if t is None:
            return
        if t.dtype != self.dtype:
            raise TypeError(f"{what}: expected {self.dtype}, got {t.dtype}")
        if tuple(t.shape) != shape or not t.is_contiguous():
            raise ValueError(f"{what}: expected a contiguous {list(shape)} tensor, got {list(t.shape)}")

    def get_params_into(self, cams_out, points_out, stream=None):
        """Copy theta into caller tensors (device or pinned host)."""
        self._check(cams_out, (self.C, 9), "cams_out")
        self._check(points_out, (self.P, 3), "points_out")
        _lib.check(_L().ba_get_params(self._h, _ptr(cams_out), _ptr(points_out), _stream(stream)))

    def set_params(self, cams=None, points=None, stream=None):
        c = None if cams is None else cams.contiguous()
        p = None if points is None else points.contiguous()
        self._check(c, (self.C, 9), "cams")
        self._check(p, (self.P, 3), "points")
        _lib.check(_L().ba_set_params(self._h, _ptr(c), _ptr(p), _stream(stream)))

    def set_pixels(self, pixels, stream=None):
        px = pixels.contiguous()
        self._check(px, (self.O, 2), "pixels")
        _lib.check(_L().ba_set_pixels(self._h, _ptr(px), _stream(stream)))

    def stats(self, cap: int = 4096, raise_nonfinite: bool = True):
        buf = (_lib.ba_iter_stats * cap)()
        n = ct.c_int()
        st = _L().ba_get_stats(self._h, buf, cap, ct.byref(n))
        out = [dict(cost=s.cost, cost_trial=s.cost_trial, model=s.model, rho=s.rho, lam=s.lambda_,
                    pcg_rel_res=s.pcg_rel_res, accepted=bool(s.accepted), pcg_iters=s.pcg_iters,
                    precond_fallbacks=s.precond_fallbacks) for s in buf[:n.value]]
        if st != _lib.BA_OK and (raise_nonfinite or st != 3):
            _lib.check(st)
        return out

    def scalars(self):
        c, l = ct.c_double(), ct.c_double()
        _lib.check(_L().ba_get_scalars(self._h, ct.byref(c), ct.byref(l)))
        return c.value, l.value

    def set_lambda(self, lam: float):
        _lib.check(_L().ba_set_lambda(self._h, float(lam)))

    def get_state(self):
        n = _L().ba_state_size(self._h)
        out = torch.empty(n, dtype=torch.float64)
        _lib.check(_L().ba_get_state(self._h, _ptr(out)))
        return out

    def set_state(self, state):
        s = torch.as_tensor(state, dtype=torch.float64).contiguous().cpu()
        if s.numel() != _L().ba_state_size(self._h):
            raise ValueError("state size mismatch")
        _lib.check(_L().ba_set_state(self._h, _ptr(s)))

    def set_fixed(self, mask=None, stream=None):
        """Freeze camera parameters: bool/uint8 [C, 9] (True = frozen) or None."""
        if mask is None:
            _lib.check(_L().ba_set_fixed(self._h, None, _stream(stream)))
            return
        m = torch.as_tensor(mask).to(device=self.device, dtype=torch.uint8).contiguous()
        if tuple(m.shape) != (self.C, 9):
            raise ValueError("mask must have shape [C, 9]")
        _lib.check(_L().ba_set_fixed(self._h, _ptr(m), _stream(stream)))
        torch.cuda.current_stream(self.device).synchronize()

    def backward(self, dL_dcams=None, dL_dpoints=None, lam: float = 0.0, maxiter: int = 1000,
                 tol: float = 1e-12, stream=None):
        """Implicit-function adjoint at the current (converged) parameters.

        Returns (dL/dpixels [O, 2], dL/dcams0 [C, 9], dL/dpoints0 [P, 3],
        pcg iterations, relative residual)."""
        def prep(t, shape):
            if t is None:
                return None
            return t.to(device=self.device, dtype=self.dtype).contiguous().reshape(shape)
        gc = prep(dL_dcams, (self.C, 9))
        gp = prep(dL_dpoints, (self.P, 3))
        dpix = torch.empty((self.O, 2), dtype=self.dtype, device=self.device)
        dc0 = torch.empty((self.C, 9), dtype=self.dtype, device=self.device)
        dp0 = torch.empty((self.P, 3), dtype=self.dtype, device=self.device)
        it = ct.c_int()
        rel = ct.c_double()
        _lib.check(_L().ba_backward(self._h, float(lam), int(maxiter), float(tol), _ptr(gc), _ptr(gp),
                                    _ptr(dpix), _ptr(dc0), _ptr(dp0), ct.byref(it), ct.byref(rel),
                                    _stream(stream)))
        return dpix, dc0, dp0, it.value, rel.value

    def layout(self):
        """Layout counts: pieces, chunks, fused_a (1/0), stored (1/0)."""
        out = (ct.c_int64 * 4)()
        _lib.check(_L().ba_get_layout(self._h, out, 4))
        names = ("pieces", "chunks", "fused_a", "stored")
        return {k: int(v) for k, v in zip(names, out)}

    def profile_trials(self, iters: int):
        """Run iters LM trials with a CUDA event pair around every launch;
        returns {kernel class: (total ms, launches)} and the trials' total ms."""
        t = _lib.ba_kernel_times()
        _lib.check(_L().ba_profile_trials(self._h, int(iters), ct.byref(t)))
        per = {name: (t.ms[i], int(t.launches[i])) for i, name in enumerate(_lib.BA_K_NAMES)}
        return per, t.trial_ms

    # -- learned block-Jacobi correction ---------------------------------------
    def set_preconditioner(self, params=None, stream=None):
        """Use the network with these parameters (FP32 [MLP_NPARAM]) for the
        PCG's block preconditioner; None returns to block-Jacobi."""
        p = None if params is None else _dev(params, torch.float32, self.device)
        if p is not None:
            _check_params(p)
        _lib.check(_L().ba_set_preconditioner(self._h, _ptr(p), _stream(stream)))
        torch.cuda.current_stream(self.device).synchronize()

    def learn_collect(self, lam: float, zhat, stream=None, scales=False):
        """Training data at the current parameters and damping lam: features
        X [C, 96], A = chol(S^_ii)^{-1} [C, 45] and y^ = S^ z^ [C, K, 9] for the
        probes zhat [C, K, 9]; with scales=True also D = diag(S_ii) [C, 9]."""
        z = _dev(zhat, torch.float32, self.device)
        K = int(z.shape[1]) if z.dim() == 3 else -1
        if K < 0 or K > _lib.BA_MLP_KMAX or tuple(z.shape) != (self.C, K, 9):
            raise ValueError(f"zhat must be [C, K, 9] with K <= {_lib.BA_MLP_KMAX}, got {list(z.shape)}")
        X = torch.empty((self.C, MLP_FIN), dtype=torch.float32, device=self.device)
        A = torch.empty((self.C, 45), dtype=torch.float32, device=self.device)
        Y = torch.empty((self.C, K, 9), dtype=torch.float32, device=self.device)
        D = torch.empty((self.C, 9), dtype=torch.float64, device=self.device) if scales else None
        _lib.check(_L().ba_learn_collect(self._h, float(lam), K, _ptr(z), _ptr(X), _ptr(A), _ptr(Y), _ptr(D),
                                         _stream(stream)))
        return (X, A, Y, D) if scales else (X, A, Y)

    def learn_slow_probes(self, lam: float, iters=(20, 50), maxiter_ref: int = 600, tol_ref: float = 1e-10,
                          stream=None):
        """Probe vectors [C, len(iters), 9] along the slow modes of the
        block-Jacobi PCG (scaled truncated-PCG errors, unit RMS)."""
        n = len(iters)
        z = torch.empty((self.C, n, 9), dtype=torch.float32, device=self.device)
        its = (ct.c_int * max(1, n))(*iters)
        _lib.check(_L().ba_learn_slow_probes(self._h, float(lam), n, ct.cast(its, ct.c_void_p), int(maxiter_ref),
                                             float(tol_ref), _ptr(z), _stream(stream)))
        return z

    # -- step-level -----------------------------------------------------------
    def csr(self, stream=None):
        d = self.device
        pc = torch.empty(self.O, dtype=torch.int32, device=d)
        rc = torch.empty(self.C + 1, dtype=torch.int32, device=d)
        pp = torch.empty(self.O, dtype=torch.int32, device=d)
        rp = torch.empty(self.P + 1, dtype=torch.int32, device=d)
        _lib.check(_L().ba_get_csr(self._h, _ptr(pc), _ptr(rc), _ptr(pp), _ptr(rp), _stream(stream)))
        return pc, rc, pp, rp

    def linearize(self, blocks=True, jacobians=True, stream=None):
        d = self.device
        f64 = torch.float64
        out = {}
        if blocks:
            out["U"] = torch.empty((self.C, 9, 9), dtype=f64, device=d)
            out["V"] = torch.empty((self.P, 3, 3), dtype=f64, device=d)
            out["gc"] = torch.empty((self.C, 9), dtype=f64, device=d)
            out["gp"] = torch.empty((self.P, 3), dtype=f64, device=d)
        if jacobians:
            out["Jc"] = torch.empty((self.O, 2, 9), dtype=self.dtype, device=d)
            out["Jp"] = torch.empty((self.O, 2, 3), dtype=self.dtype, device=d)
            out["w"] = torch.empty((self.O,), dtype=self.dtype, device=d)
        g = out.get
        _lib.check(_L().ba_linearize(self._h, _ptr(g("U")), _ptr(g("V")), _ptr(g("gc")),
                                     _ptr(g("gp")), _ptr(g("Jc")), _ptr(g("Jp")), _ptr(g("w")),
                                     _stream(stream)))
        return out

    def schur_matvec(self, lam: float, x, stream=None):
        x = x.to(device=self.device, dtype=torch.float64).contiguous()
        y = torch.empty_like(x)
        _lib.check(_L().ba_schur_matvec(self._h, float(lam), _ptr(x), _ptr(y), _stream(stream)))
        return y

    def damped_solve(self, lam: float, maxiter: int, tol: float, stream=None):
        dc = torch.empty((self.C, 9), dtype=torch.float64, device=self.device)
        dp = torch.empty((self.P, 3), dtype=self.dtype, device=self.device)
        it = ct.c_int()
        rel = ct.c_double()
        _lib.check(_L().ba_damped_solve(self._h, float(lam), int(maxiter), float(tol), _ptr(dc),
                                        _ptr(dp), ct.byref(it), ct.byref(rel), _stream(stream)))
        return dc, dp, it.value, rel.value


def _stats_dict(s):
    return dict(cost=s.cost, cost_trial=s.cost_trial, model=s.model, rho=s.rho, lam=s.lambda_,
                pcg_rel_res=s.pcg_rel_res, accepted=bool(s.accepted), pcg_iters=s.pcg_iters,
                precond_fallbacks=s.precond_fallbacks)


class Batch:
    """Many independent small problems solved by one persistent launch.

    problems: a sequence of (cams [C_b, 9], points [P_b, 3], cam_idx [O_b],
    pt_idx [O_b], pixels [O_b, 2]) with indices local to the problem;
    C_b <= 28 and every point observed.  Each problem runs exactly the trials
    a Problem of its own would run with the same options."""

    MAX_CAMS = _lib.BA_BATCH_MAX_CAMS

    def __init__(self, problems, options: Options | None = None, device="cuda", stream=None):
        self.options = options or Options()
        self.dtype = self.options.dtype
        self.device = torch.device(device)
        problems = list(problems)
        if not problems:
            raise ValueError("empty batch")
        cams = [torch.as_tensor(p[0]) for p in problems]
        pts = [torch.as_tensor(p[1]) for p in problems]
        ci = [torch.as_tensor(p[2]) for p in problems]
        pi = [torch.as_tensor(p[3]) for p in problems]
        px = [torch.as_tensor(p[4]) for p in problems]
        for arrays in zip(cams, pts, ci, pi, px):
            _check_problem_shapes(*arrays)
        self.n = len(problems)
        self.cam_counts = [int(c.shape[0]) for c in cams]
        self.pt_counts = [int(p.shape[0]) for p in pts]
        self.obs_counts = [int(c.shape[0]) for c in ci]
        cat = lambda xs, dt: _dev(torch.cat([x.reshape(x.shape[0], -1) if x.dim() > 1 else x for x in xs]), dt,
                                  self.device)
        c_all = cat(cams, self.dtype)
        p_all = cat(pts, self.dtype)
        ci_all = cat(ci, torch.int32)
        pi_all = cat(pi, torch.int32)
        px_all = cat(px, self.dtype)
        self.C, self.P, self.O = int(c_all.shape[0]), int(p_all.shape[0]), int(ci_all.shape[0])
        counts = [(ct.c_int32 * self.n)(*v) for v in (self.cam_counts, self.pt_counts, self.obs_counts)]
        h = ct.c_void_p()
        o = self.options.to_c()
        _lib.check(_L().ba_batch_create(ct.byref(h), self.n, ct.cast(counts[0], ct.c_void_p),
                                        ct.cast(counts[1], ct.c_void_p), ct.cast(counts[2], ct.c_void_p),
                                        _ptr(c_all), _ptr(p_all), _ptr(ci_all), _ptr(pi_all), _ptr(px_all),
                                        ct.byref(o), _stream(stream)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _L().ba_batch_destroy(self._h)
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
        _lib.check(_L().ba_batch_solve(self._h, int(iters), _stream(stream)))

    def params(self, stream=None, split: bool = True):
        cams = torch.empty((self.C, 9), dtype=self.dtype, device=self.device)
        pts = torch.empty((self.P, 3), dtype=self.dtype, device=self.device)
        _lib.check(_L().ba_batch_get_params(self._h, _ptr(cams), _ptr(pts), _stream(stream)))
        if not split:
            return cams, pts
        return list(zip(torch.split(cams, self.cam_counts), torch.split(pts, self.pt_counts)))

    def reset(self, cams=None, points=None, stream=None):
        c = None if cams is None else _dev(cams, self.dtype, self.device)
        p = None if points is None else _dev(points, self.dtype, self.device)
        for t, shape, what in ((c, (self.C, 9), "cams"), (p, (self.P, 3), "points")):
            if t is not None and tuple(t.shape) != shape:
                raise ValueError(f"{what}: expected the concatenated {list(shape)}, got {list(t.shape)}")
        _lib.check(_L().ba_batch_reset(self._h, _ptr(c), _ptr(p), _stream(stream)))

    def stats(self, cap: int = 256, raise_nonfinite: bool = True):
        buf = (_lib.ba_iter_stats * (cap * self.n))()
        n = (ct.c_int * self.n)()
        st = _L().ba_batch_get_stats(self._h, buf, cap, ct.cast(n, ct.c_void_p))
        out = [[_stats_dict(buf[b * cap + k]) for k in range(n[b])] for b in range(self.n)]
        if st != _lib.BA_OK and (raise_nonfinite or st != 3):
            _lib.check(st)
        return out

    def scalars(self):
        cost = (ct.c_double * self.n)()
        lam = (ct.c_double * self.n)()
        _lib.check(_L().ba_batch_get_scalars(self._h, ct.cast(cost, ct.c_void_p), ct.cast(lam, ct.c_void_p)))
        return list(cost), list(lam)

    def set_launch(self, ctas_per_sm: int, variant: int = 0, order: int = 0):
        _lib.check(_L().ba_batch_set_launch(self._h, int(ctas_per_sm), int(variant), int(order)))

    def launch(self):
        c, v, o, g = ct.c_int(), ct.c_int(), ct.c_int(), ct.c_int()
        _lib.check(_L().ba_batch_get_launch(self._h, ct.byref(c), ct.byref(v), ct.byref(o), ct.byref(g)))
        return dict(ctas_per_sm=c.value, variant=v.value, order=o.value, grid=g.value)

    def set_segments(self, piece_max: int = 2048, chunk_slots: int = 1024, chunk_pts: int = 512):
        """Segment sizes of the solve (pieces of camera-major slots, point
        chunks); another cut moves results by rounding."""
        _lib.check(_L().ba_batch_set_segments(self._h, int(piece_max), int(chunk_slots), int(chunk_pts)))

    def segments(self):
        p, s, t = ct.c_int(), ct.c_int(), ct.c_int()
        _lib.check(_L().ba_batch_get_segments(self._h, ct.byref(p), ct.byref(s), ct.byref(t)))
        return dict(piece_max=p.value, chunk_slots=s.value, chunk_pts=t.value)

    def autotune(self, iters: int, cache_path: str | None = None):
        """Pick the fastest launch configuration (results do not depend on
        it), then the fastest segment sizes whose final costs stay within
        1e-6 of the current ones; returns the chosen launch and segments and
        the time (0 if cached)."""
        ms = ct.c_double()
        path = None if cache_path is None else str(cache_path).encode()
        _lib.check(_L().ba_batch_autotune(self._h, int(iters), path, ct.byref(ms)))
        return {**self.launch(), **self.segments()}, ms.value


class _BundleAdjust(torch.autograd.Function):
    """theta* = LM(pixels, theta0) with the implicit-function adjoint as its
    backward (gradients w.r.t. the observed pixels and the initial
    parameters)."""

    @staticmethod
    def forward(ctx, pixels, cams0, points0, problem, iters, adjoint):
        problem.set_params(cams0.detach().to(problem.dtype).contiguous(),
                           points0.detach().to(problem.dtype).contiguous())
        problem.set_pixels(pixels.detach().to(problem.dtype).contiguous())
        problem.set_lambda(problem.options.lambda0)
        problem.solve(iters)
        cams, points = problem.params()
        ctx.problem = problem
        ctx.adjoint = adjoint
        ctx.dtypes = (pixels.dtype, cams0.dtype, points0.dtype)
        return cams, points

    @staticmethod
    def backward(ctx, g_cams, g_points):
        dpix, dc0, dp0, _, _ = ctx.problem.backward(g_cams, g_points, **ctx.adjoint)
        tp, tc, tq = ctx.dtypes
        return dpix.to(tp), dc0.to(tc), dp0.to(tq), None, None, None


def bundle_adjust(pixels, cams0, points0, problem: "Problem", iters: int, lam: float = 0.0,
                  maxiter: int = 1000, tol: float = 1e-12):
    """Differentiable LM solve on an existing problem (its structure and
    frozen-parameter mask are reused): returns (cams*, points*); gradients
    flow to pixels, cams0 and points0 through the implicit-function adjoint."""
    return _BundleAdjust.apply(pixels, cams0, points0, problem, int(iters),
                               dict(lam=lam, maxiter=maxiter, tol=tol))


def project(cams, points, cam_idx, pt_idx, stream=None):
    """pi(theta_c(k), X_p(k)) for every observation (device tensors)."""
    if cams.dtype not in (torch.float32, torch.float64) or points.dtype != cams.dtype:
        raise TypeError("cams and points must share a float32/float64 dtype")
    prec = BA_PREC_F32 if cams.dtype == torch.float32 else BA_PREC_F64
    cams, points = cams.contiguous(), points.contiguous()
    ci = cam_idx.to(torch.int32).contiguous()
    pi = pt_idx.to(torch.int32).contiguous()
    if cams.dim() != 2 or cams.shape[1] != 9 or points.dim() != 2 or points.shape[1] != 3 or \
            ci.dim() != 1 or tuple(pi.shape) != tuple(ci.shape):
        raise ValueError("project: cams [C, 9], points [P, 3], cam_idx and pt_idx [O]")
    out = torch.empty((ci.shape[0], 2), dtype=cams.dtype, device=cams.device)
    _lib.check(_L().ba_project(prec, cams.shape[0], points.shape[0], ci.shape[0], _ptr(cams),
                               _ptr(points), _ptr(ci), _ptr(pi), _ptr(out), _stream(stream)))
    return out


def csr_build(keys, n_keys: int, stream=None):
    """Stable sort of int32 device keys in [0, n_keys): (perm, rowptr)."""
    k = keys.to(torch.int32).contiguous()
    perm = torch.empty(k.shape[0], dtype=torch.int32, device=k.device)
    rowptr = torch.empty(n_keys + 1, dtype=torch.int32, device=k.device)
    _lib.check(_L().ba_csr_build(_ptr(k) if k.numel() else None, k.shape[0], int(n_keys),
                                 _ptr(perm) if k.numel() else None, _ptr(rowptr), _stream(stream)))
    return perm, rowptr


def _check_params(params):
    if params.dtype != torch.float32 or params.numel() != MLP_NPARAM or not params.is_contiguous():
        raise ValueError(f"network parameters must be a contiguous float32 [{MLP_NPARAM}] tensor")


def _check_samples(X, A=None, Y=None, Z=None):
    """Sample arrays of the learned correction: X [n, 96], A [n, 45],
    Y and Z [n, K, 9] with K <= BA_MLP_KMAX (sizes the library cannot see)."""
    n = int(X.shape[0])
    if tuple(X.shape) != (n, MLP_FIN):
        raise ValueError(f"X must be [n, {MLP_FIN}], got {list(X.shape)}")
    if A is not None and tuple(A.shape) != (n, MLP_FOUT):
        raise ValueError(f"A must be [n, {MLP_FOUT}], got {list(A.shape)}")
    if Y is not None:
        K = int(Y.shape[1]) if Y.dim() == 3 else -1
        if K < 0 or K > _lib.BA_MLP_KMAX or tuple(Y.shape) != (n, K, 9) or tuple(Z.shape) != (n, K, 9):
            raise ValueError(f"Y and Z must be [n, K, 9] with K <= {_lib.BA_MLP_KMAX}, "
                             f"got {list(Y.shape)}, {list(Z.shape)}")


def mlp_init(seed: int = 0, device="cuda"):
    """Initial network parameters (FP32 [MLP_NPARAM]): uniform +-1/sqrt(fan_in)
    weights and biases in the hidden layers, a zero output layer (so the
    preconditioner starts as block-Jacobi)."""
    g = torch.Generator().manual_seed(int(seed))
    parts = []
    for fan_out, fan_in, zero in ((64, MLP_FIN, False), (64, 64, False), (MLP_FOUT, 64, True)):
        bound = 1.0 / fan_in ** 0.5
        w = torch.zeros(fan_out * fan_in) if zero else (torch.rand(fan_out * fan_in, generator=g) * 2 - 1) * bound
        b = torch.zeros(fan_out) if zero else (torch.rand(fan_out, generator=g) * 2 - 1) * bound
        parts += [w, b]
    return torch.cat(parts).to(device=device, dtype=torch.float32)


def mlp_forward(params, X, stream=None):
    """Network output [n, 45] for features X [n, 96] (tensor-core kernel)."""
    X = X.to(torch.float32).contiguous()
    params = params.contiguous()
    _check_params(params)
    _check_samples(X)
    E = torch.empty((X.shape[0], MLP_FOUT), dtype=torch.float32, device=X.device)
    _lib.check(_L().ba_mlp_forward(_ptr(params), int(X.shape[0]), _ptr(X), _ptr(E), _stream(stream)))
    return E


def mlp_loss_grad(params, X, A, Y, Z, stream=None):
    """(mean probe loss, gradient [MLP_NPARAM] float64)."""
    _check_samples(X, A, Y, Z)
    params = params.contiguous()
    _check_params(params)
    n, K = int(X.shape[0]), int(Y.shape[1])
    grad = torch.empty(MLP_NPARAM, dtype=torch.float64, device=X.device)
    loss = ct.c_double()
    args = [t.to(torch.float32).contiguous() for t in (X, A, Y, Z)]
    _lib.check(_L().ba_mlp_loss_grad(_ptr(params), n, K, *(_ptr(t) for t in args), _ptr(grad),
                                     ct.byref(loss), _stream(stream)))
    return loss.value, grad


def mlp_train(params, adam_m, adam_v, X, A, Y, Z, epochs: int, batch: int, lr: float, stream=None):
    """Adam on params (in place, FP32 device tensors) over minibatches of
    consecutive samples; returns the per-epoch mean minibatch losses."""
    _check_samples(X, A, Y, Z)
    n, K = int(X.shape[0]), int(Y.shape[1])
    hist = (ct.c_double * max(1, int(epochs)))()
    args = [t.to(torch.float32).contiguous() for t in (X, A, Y, Z)]
    for t in (params, adam_m, adam_v):
        if not (t.is_contiguous() and t.dtype == torch.float32 and t.numel() == MLP_NPARAM):
            raise ValueError("params / moments must be contiguous float32 [MLP_NPARAM]")
    _lib.check(_L().ba_mlp_train(_ptr(params), _ptr(adam_m), _ptr(adam_v), n, K, *(_ptr(t) for t in args),
                                 int(epochs), int(batch), float(lr), ct.cast(hist, ct.c_void_p),
                                 _stream(stream)))
    return list(hist)[:int(epochs)]


def measure_fma_peak(precision: str = "f64", stream=None) -> float:
    """Measured FMA throughput of the CUDA cores in TFLOP/s ("f64" or "f32")."""
    if precision not in ("f32", "f64"):
        raise ValueError("precision must be 'f32' or 'f64'")
    out = ct.c_double()
    _lib.check(_L().ba_measure_fma_peak(BA_PREC_F32 if precision == "f32" else BA_PREC_F64, ct.byref(out),
                                        _stream(stream)))
    return out.value


def kernel_launch_count() -> int:
    return int(_L().ba_kernel_launch_count())


from .pgo import PoseGraph  # noqa: E402  (needs the helpers above)
