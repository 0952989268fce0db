"""A C99 program solves ba16 through include/ba.h with host pointers only
(no CUDA headers, no Python in the solving process); its per-trial costs
and final cameras match the oracle's LM with a Cholesky solve of the
reduced system (the GPU runs PCG to 1e-14, at most 9C iterations)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as orc
import scenegen

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _write_problem(path, sc, pix, iters, pcg_maxiter, pcg_tol):
    with open(path, "wb") as f:
        np.array([sc.C, sc.P, sc.O, iters, pcg_maxiter], dtype=np.int32).tofile(f)
        np.array([pcg_tol], dtype=np.float64).tofile(f)
        np.ascontiguousarray(sc.cams_init, dtype=np.float64).tofile(f)
        np.ascontiguousarray(sc.points_init, dtype=np.float64).tofile(f)
        np.ascontiguousarray(sc.cam_idx, dtype=np.int32).tofile(f)
        np.ascontiguousarray(sc.pt_idx, dtype=np.int32).tofile(f)
        np.ascontiguousarray(pix, dtype=np.float64).tofile(f)


def test_c_program_solve_matches_oracle(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_2409_12190_gb300 import build as b
    libdir = os.path.dirname(b.build())
    exe = tmp_path / "solve_from_c"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "solve_from_c.c"), "-L", libdir, "-lba_gb300",
                    f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    sc = scenegen.config_scene("ba16")
    pix = orc.pixels_from_scene(sc)
    iters = 12
    prob = tmp_path / "ba16.bin"
    _write_problem(prob, sc, pix, iters, 9 * sc.C, 1e-14)
    out = subprocess.run([str(exe), str(prob)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    lines = out.stdout.split("\n")
    trials = [ln.split() for ln in lines if ln.startswith("trial ")]
    cams = np.array([float(ln.split()[1]) for ln in lines if ln.startswith("cam ")]).reshape(sc.C, 9)
    cams_ref, _, ref = orc.lm(sc.cams_init, sc.points_init, sc.cam_idx, sc.pt_idx, pix, iters,
                              orc.LMOptions(solver="cholesky"))
    assert len(trials) == iters
    for t, r in zip(trials, ref):
        assert abs(float(t[2]) - r["cost"]) <= 1e-9 * r["cost"], (t, r)
        assert abs(float(t[3]) - r["cost_trial"]) <= 1e-9 * r["cost_trial"], (t, r)
        if abs(r["cost"] - r["cost_trial"]) > 1e-7 * r["cost"]:
            assert bool(int(t[4])) == r["accepted"], (t, r)
    scale = np.maximum(1.0, np.abs(cams_ref))
    assert np.max(np.abs(cams - cams_ref) / scale) < 1e-7
