"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/ba.h declares (no compute calls)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2409_12190_gb300 import build as b
    path = b.build()
    return ctypes.CDLL(path)


def _declared():
    src = open(os.path.join(ROOT, "include", "ba.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ba_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("ba_problem_create", "ba_lm_step", "ba_solve", "ba_get_params", "ba_get_stats",
              "ba_problem_destroy", "ba_last_error", "ba_csr_build", "ba_project"):
        assert n in names


def test_every_declaration_cites_the_paper_or_says_it_has_no_counterpart():
    """Each entry point's comment names the passage it implements (Sec., Eq.,
    Alg., App.) or states that the paper has no counterpart."""
    lines = open(os.path.join(ROOT, "include", "ba.h")).read().split("\n")
    decl = re.compile(r"^(ba_status|const char\*|size_t|uint64_t)\s+(ba_[a-z_0-9]+)\s*\(")
    cite = re.compile(r"Sec\.|Eq\.|Alg\.|App\.|no counterpart|[Nn]ot in the paper")
    missing = []
    for i, line in enumerate(lines):
        m = decl.match(line)
        if not m:
            continue
        j, comment = i - 1, []
        while j >= 0 and lines[j].strip().startswith(("/*", "*")) or (j >= 0 and lines[j].strip().endswith("*/")):
            comment.insert(0, lines[j])
            j -= 1
        if not cite.search(" ".join(comment)):
            missing.append(m.group(2))
    assert not missing, missing


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    from paper_2409_12190_gb300 import _lib
    assert set(_declared()) <= set(_lib.SIGNATURES)


def test_options_default_without_gpu(lib):
    from paper_2409_12190_gb300 import _lib
    L = _lib.load()
    o = _lib.ba_options()
    assert L.ba_options_default(ctypes.byref(o)) == 0
    assert o.up == 2.0 and o.down == 0.0625 and o.pcg_maxiter == 250 and o.pcg_tol == 1e-4
    assert o.lambda0 == 1e-4 and o.diag_min == 1e-6


def test_struct_layouts_match_header():
    from paper_2409_12190_gb300 import _lib
    assert ctypes.sizeof(_lib.ba_iter_stats) == 6 * 8 + 4 * 4
    # int (+pad), 10 doubles, int (+pad), double, 3 ints (+pad)
    assert ctypes.sizeof(_lib.ba_options) == 8 + 80 + 8 + 8 + 16


def test_argument_errors_need_no_gpu(lib):
    from paper_2409_12190_gb300 import _lib
    L = _lib.load()
    h = ctypes.c_void_p()
    assert L.ba_problem_create(ctypes.byref(h), 0, 1, 1, None, None, None, None, None, None, None) == 1
    assert b"must be >= 1" in L.ba_last_error()
    assert L.ba_csr_build(None, -1, 3, None, None, None) == 1
    assert L.ba_lm_step(None, None) == 1


def test_batch_argument_errors_need_no_gpu(lib):
    from paper_2409_12190_gb300 import _lib
    L = _lib.load()
    h = ctypes.c_void_p()
    dummy = ctypes.c_void_p(256)  # never dereferenced: the counts are checked first
    one = (ctypes.c_int32 * 1)(1)
    too_many = (ctypes.c_int32 * 1)(_lib.BA_BATCH_MAX_CAMS + 1)
    assert L.ba_batch_create(ctypes.byref(h), 0, one, one, one, dummy, dummy, dummy, dummy, dummy, None,
                             None) == 1
    assert b"nprob" in L.ba_last_error()
    assert L.ba_batch_create(ctypes.byref(h), 1, too_many, one, one, dummy, dummy, dummy, dummy, dummy, None,
                             None) == 1
    assert b"C_b" in L.ba_last_error()
    assert L.ba_batch_solve(None, 1, None) == 1
    assert L.ba_batch_set_launch(None, 1, 0, 0) == 1


def test_batch_max_cams_matches_header():
    from paper_2409_12190_gb300 import _lib
    src = open(os.path.join(ROOT, "include", "ba.h")).read()
    m = re.search(r"#define BA_BATCH_MAX_CAMS (\d+)", src)
    assert m and int(m.group(1)) == _lib.BA_BATCH_MAX_CAMS


def test_plain_c_program_uses_the_header_and_library(lib, tmp_path):
    """The boundary needs neither Python nor torch: a C99 program compiled
    against include/ba.h and linked to the library reads the defaults and
    gets the documented argument errors (no GPU work)."""
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    libdir = os.path.dirname(lib._name)
    exe = tmp_path / "abi_from_c"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "abi_from_c.c"), "-L", libdir, "-lba_gb300",
                    f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "OK", out.stderr


@pytest.mark.parametrize("bad", ["cams", "points", "pt_idx", "pixels"])
def test_binding_rejects_mismatched_shapes_before_any_library_call(bad):
    """The C ABI sees plain pointers; the binding checks shapes on the host,
    so a wrong shape is a ValueError and never a read past a buffer's end."""
    import numpy as np
    import paper_2409_12190_gb300 as ba
    C, P, O = 3, 5, 7
    arrays = dict(cams=np.zeros((C, 9)), points=np.zeros((P, 3)), cam_idx=np.zeros(O, np.int32),
                  pt_idx=np.zeros(O, np.int32), pixels=np.zeros((O, 2)))
    arrays[bad] = {"cams": np.zeros((C, 8)), "points": np.zeros((P, 2)), "pt_idx": np.zeros(O - 1, np.int32),
                   "pixels": np.zeros((O - 1, 2))}[bad]
    with pytest.raises(ValueError):
        ba.Problem(arrays["cams"], arrays["points"], arrays["cam_idx"], arrays["pt_idx"], arrays["pixels"],
                   device="cpu")
    with pytest.raises(ValueError):
        ba.Batch([(arrays["cams"], arrays["points"], arrays["cam_idx"], arrays["pt_idx"], arrays["pixels"])],
                 device="cpu")


def test_project_rejects_mismatched_index_lengths():
    import torch
    import paper_2409_12190_gb300 as ba
    with pytest.raises(ValueError):
        ba.project(torch.zeros(3, 9, dtype=torch.float64), torch.zeros(5, 3, dtype=torch.float64),
                   torch.zeros(7, dtype=torch.int32), torch.zeros(6, dtype=torch.int32))


def test_learned_correction_bindings_reject_wrong_sizes():
    import torch
    import paper_2409_12190_gb300 as ba
    p = torch.zeros(ba.MLP_NPARAM)
    X = torch.zeros(4, ba.MLP_FIN)
    A = torch.zeros(4, 45)
    Y = torch.zeros(4, 2, 9)
    with pytest.raises(ValueError):
        ba.mlp_forward(p[:-1], X)                        # parameters too short
    with pytest.raises(ValueError):
        ba.mlp_forward(p.double(), X)                    # wrong parameter dtype
    with pytest.raises(ValueError):
        ba.mlp_forward(p, X[:, :-1])                     # features too narrow
    with pytest.raises(ValueError):
        ba.mlp_loss_grad(p, X, A[:3], Y, Y)              # A of another sample count
    with pytest.raises(ValueError):
        ba.mlp_loss_grad(p, X, A, Y, Y[:, :1])           # Z with other probes than Y
    with pytest.raises(ValueError):
        ba.mlp_loss_grad(p, X, A, torch.zeros(4, 17, 9), torch.zeros(4, 17, 9))   # K > BA_MLP_KMAX
    with pytest.raises(ValueError):
        ba.mlp_train(p, p.clone(), p.clone(), X, A, Y, Y[:3], epochs=1, batch=4, lr=1e-3)
