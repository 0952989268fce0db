"""Constants the paper prints (tests/golden/, each file names its source):
the oracle's LM defaults and the C ABI's defaults must be those values."""
import ctypes
import json
import os

import oracle as orc

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_oracle_defaults_are_the_papers_solver_constants():
    g = _load("paper_solver_constants.json")
    o = orc.LMOptions()
    assert (o.pcg_tol, o.pcg_maxiter) == (g["pcg_tol"], g["pcg_maxiter"])
    assert (o.up, o.down) == (g["trust_region_up"], g["trust_region_down"])
    assert g["trust_region_down"] == 0.5 ** 4


def test_library_defaults_are_the_papers_solver_constants():
    g = _load("paper_solver_constants.json")
    from paper_2409_12190_gb300 import _lib
    L = _lib.load()
    o = _lib.ba_options()
    assert L.ba_options_default(ctypes.byref(o)) == 0
    assert (o.pcg_tol, o.pcg_maxiter) == (g["pcg_tol"], g["pcg_maxiter"])
    assert (o.up, o.down) == (g["trust_region_up"], g["trust_region_down"])
