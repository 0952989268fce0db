"""ctypes declarations of the C ABI in include/ba.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as ct
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libba_gb300.so")

BA_OK = 0
STATUS_NAMES = {0: "BA_OK", 1: "BA_ERR_INVALID_ARG", 2: "BA_ERR_CUDA", 3: "BA_ERR_NONFINITE",
                4: "BA_ERR_TIMEOUT", 5: "BA_ERR_NOT_CONVERGED", 6: "BA_ERR_OOM", 7: "BA_ERR_STATE"}
BA_PREC_F64 = 0
BA_PREC_F32 = 1
BA_JAC = {"auto": 0, "recompute": 1, "store": 2}
BA_SOLVER = {"pcg": 0, "cholesky": 1}


class ba_options(ct.Structure):
    _fields_ = [
        ("precision", ct.c_int),
        ("huber_delta", ct.c_double),
        ("lambda0", ct.c_double),
        ("up", ct.c_double),
        ("down", ct.c_double),
        ("rho_good", ct.c_double),
        ("rho_bad", ct.c_double),
        ("lambda_min", ct.c_double),
        ("lambda_max", ct.c_double),
        ("diag_min", ct.c_double),
        ("diag_max", ct.c_double),
        ("pcg_maxiter", ct.c_int),
        ("pcg_tol", ct.c_double),
        ("use_graph", ct.c_int),
        ("max_stats", ct.c_int),
        ("jacobian_mode", ct.c_int),
        ("solver", ct.c_int),
    ]


class ba_iter_stats(ct.Structure):
    _fields_ = [
        ("cost", ct.c_double),
        ("cost_trial", ct.c_double),
        ("model", ct.c_double),
        ("rho", ct.c_double),
        ("lambda_", ct.c_double),
        ("pcg_rel_res", ct.c_double),
        ("accepted", ct.c_int32),
        ("pcg_iters", ct.c_int32),
        ("precond_fallbacks", ct.c_int32),
        ("reserved", ct.c_int32),
    ]


BA_K_NAMES = ["lin_cam", "lin_pt", "schur_cam", "pass_a1", "pass_b", "cost", "backsub", "other", "pass_a2",
              "pass_fa"]


class ba_kernel_times(ct.Structure):
    _fields_ = [("ms", ct.c_double * 10), ("launches", ct.c_int64 * 10), ("trial_ms", ct.c_double)]


_VP = ct.c_void_p
_I = ct.c_int
_D = ct.c_double
_S = ct.c_int  # ba_status

# ba_exchange_fn: int (*)(size_t n, void* stream, void* ctx)
EXCHANGE_FN = ct.CFUNCTYPE(ct.c_int, ct.c_size_t, ct.c_void_p, ct.c_void_p)

# name -> (restype, argtypes)
SIGNATURES = {
    "ba_options_default": (_S, [ct.POINTER(ba_options)]),
    "ba_problem_create": (_S, [ct.POINTER(_VP), _I, _I, _I, _VP, _VP, _VP, _VP, _VP,
                               ct.POINTER(ba_options), _VP]),
    "ba_problem_destroy": (_S, [_VP]),
    "ba_lm_step": (_S, [_VP, _VP]),
    "ba_solve": (_S, [_VP, _I, _VP]),
    "ba_get_params": (_S, [_VP, _VP, _VP, _VP]),
    "ba_set_params": (_S, [_VP, _VP, _VP, _VP]),
    "ba_set_pixels": (_S, [_VP, _VP, _VP]),
    "ba_get_stats": (_S, [_VP, ct.POINTER(ba_iter_stats), _I, ct.POINTER(_I)]),
    "ba_get_scalars": (_S, [_VP, ct.POINTER(_D), ct.POINTER(_D)]),
    "ba_state_size": (ct.c_size_t, [_VP]),
    "ba_get_state": (_S, [_VP, _VP]),
    "ba_set_state": (_S, [_VP, _VP]),
    "ba_last_error": (ct.c_char_p, []),
    "ba_get_csr": (_S, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "ba_linearize": (_S, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "ba_schur_matvec": (_S, [_VP, _D, _VP, _VP, _VP]),
    "ba_damped_solve": (_S, [_VP, _D, _I, _D, _VP, _VP, ct.POINTER(_I), ct.POINTER(_D), _VP]),
    "ba_project": (_S, [_I, _I, _I, _I, _VP, _VP, _VP, _VP, _VP, _VP]),
    "ba_csr_build": (_S, [_VP, _I, _I, _VP, _VP, _VP]),
    "ba_csr_build_noalloc": (_S, [_VP, _I, _I, _VP, _VP, _VP]),
    "ba_kernel_launch_count": (ct.c_uint64, []),
    "ba_profile_trials": (_S, [_VP, _I, ct.POINTER(ba_kernel_times)]),
    "ba_measure_fma_peak": (_S, [_I, ct.POINTER(_D), _VP]),
    "ba_get_layout": (_S, [_VP, _VP, _I]),
    "ba_set_exchange": (_S, [_VP, EXCHANGE_FN, _VP, _VP, ct.c_size_t]),
    "ba_set_fixed": (_S, [_VP, _VP, _VP]),
    "ba_set_lambda": (_S, [_VP, _D]),
    "ba_backward": (_S, [_VP, _D, _I, _D, _VP, _VP, _VP, _VP, _VP, ct.POINTER(_I), ct.POINTER(_D), _VP]),
    "ba_batch_create": (_S, [ct.POINTER(_VP), _I, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                             ct.POINTER(ba_options), _VP]),
    "ba_batch_destroy": (_S, [_VP]),
    "ba_batch_solve": (_S, [_VP, _I, _VP]),
    "ba_batch_get_params": (_S, [_VP, _VP, _VP, _VP]),
    "ba_batch_reset": (_S, [_VP, _VP, _VP, _VP]),
    "ba_batch_get_stats": (_S, [_VP, ct.POINTER(ba_iter_stats), _I, _VP]),
    "ba_batch_get_scalars": (_S, [_VP, _VP, _VP]),
    "ba_batch_set_launch": (_S, [_VP, _I, _I, _I]),
    "ba_batch_get_launch": (_S, [_VP, ct.POINTER(_I), ct.POINTER(_I), ct.POINTER(_I), ct.POINTER(_I)]),
    "ba_batch_autotune": (_S, [_VP, _I, ct.c_char_p, ct.POINTER(_D)]),
    "ba_batch_set_segments": (_S, [_VP, _I, _I, _I]),
    "ba_batch_get_segments": (_S, [_VP, ct.POINTER(_I), ct.POINTER(_I), ct.POINTER(_I)]),
    "ba_set_preconditioner": (_S, [_VP, _VP, _VP]),
    "ba_learn_collect": (_S, [_VP, _D, _I, _VP, _VP, _VP, _VP, _VP, _VP]),
    "ba_learn_slow_probes": (_S, [_VP, _D, _I, _VP, _I, _D, _VP, _VP]),
    "ba_mlp_forward": (_S, [_VP, _I, _VP, _VP, _VP]),
    "ba_mlp_loss_grad": (_S, [_VP, _I, _I, _VP, _VP, _VP, _VP, _VP, ct.POINTER(_D), _VP]),
    "ba_mlp_train": (_S, [_VP, _VP, _VP, _I, _I, _VP, _VP, _VP, _VP, _I, _I, _D, _VP, _VP]),
    "ba_pgo_create": (_S, [ct.POINTER(_VP), _I, _I, _VP, _VP, _VP, _VP, _VP, _VP, ct.POINTER(ba_options), _VP]),
    "ba_pgo_destroy": (_S, [_VP]),
    "ba_pgo_solve": (_S, [_VP, _I, _VP]),
    "ba_pgo_get_poses": (_S, [_VP, _VP, _VP]),
    "ba_pgo_set_poses": (_S, [_VP, _VP, _VP]),
    "ba_pgo_get_stats": (_S, [_VP, ct.POINTER(ba_iter_stats), _I, ct.POINTER(_I)]),
    "ba_pgo_get_scalars": (_S, [_VP, ct.POINTER(_D), ct.POINTER(_D)]),
    "ba_pgo_set_lambda": (_S, [_VP, _D]),
    "ba_pgo_linearize": (_S, [_VP, _VP, _VP, _VP, _VP, _VP, ct.POINTER(_D), _VP]),
    "ba_pgo_matvec": (_S, [_VP, _D, _VP, _VP, _VP]),
    "ba_pgo_damped_solve": (_S, [_VP, _D, _I, _D, _VP, ct.POINTER(_I), ct.POINTER(_D), _VP]),
    "ba_pgo_synthesize": (_S, [_I, _I, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
}

BA_MLP_FIN = 96
BA_MLP_FOUT = 45
BA_MLP_NPARAM = 13293
BA_MLP_KMAX = 16

BA_BATCH_MAX_CAMS = 28

_lib = None


def load(path: str | None = None):
    """Load the shared library; raises if it has not been built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(
            f"{p} not found: build it first with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (nvcc, sm_103a)")
    lib = ct.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


class BAError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int):
    if status != BA_OK:
        raise BAError(status, load().ba_last_error().decode(errors="replace"))
