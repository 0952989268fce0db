"""Build the sm_103a shared library ``libba_gb300.so`` in-tree with nvcc.

Each translation unit is compiled in parallel, then linked with the static
CUDA runtime.  Re-running is cheap: a unit is rebuilt only when a source or
header is newer than its object.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libba_gb300.so")
UNITS = ["ba_api.cu", "ba_sort.cu", "ba_noalloc.cu", "ba_batch.cu", "ba_learn.cu", "ba_measure.cu", "ba_pgo.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(extra=()):
    return ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
            "-I", INCLUDE, "-I", CSRC, *extra]


def _deps_mtime():
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "ba.h")]
    return max(os.path.getmtime(p) for p in paths)


def build(verbose: bool = False, ptxas_verbose: bool = False, force: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = nvcc_path()
    newest = _deps_mtime()
    extra = ["-Xptxas", "-v"] if ptxas_verbose else []

    def compile_unit(unit):
        obj = os.path.join(BUILD, unit.replace(".cu", ".o"))
        if not force and not ptxas_verbose and os.path.exists(obj) and os.path.getmtime(obj) >= newest:
            return obj, ""
        # a per-process temporary, then an atomic rename: processes that
        # build at the same time (the ranks of one job) never see a torn file
        tmp_obj = f"{obj}.{os.getpid()}.tmp"
        cmd = [nvcc, *_flags(extra), "-c", os.path.join(CSRC, unit), "-o", tmp_obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed for {unit}:\n{' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
        os.replace(tmp_obj, obj)
        return obj, res.stdout + res.stderr

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        results = list(ex.map(compile_unit, UNITS))
    logs = "".join(r[1] for r in results)
    objs = [r[0] for r in results]
    if force or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = f"{LIB}.{os.getpid()}.tmp"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
        os.replace(tmp, LIB)
    if verbose and logs:
        sys.stdout.write(logs)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, ptxas_verbose="-v" in sys.argv, force="-f" in sys.argv))
