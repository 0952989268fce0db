"""a0: the symbolic phase (stable sort + row pointers) is bit-exact with the
oracle's counting sort."""
import numpy as np
import pytest
import torch

import oracle as orc
import paper_2409_12190_gb300 as ba
import scenegen
from gpu_helpers import problem

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,K", [(0, 1), (1, 1), (5, 1), (1000, 3), (4096, 17), (4097, 300),
                                 (8191, 256), (8192, 257), (100_000, 1_200_000), (300_000, 70_000),
                                 (65_536, 65_536)])
def test_csr_build_standalone(n, K):
    rng = np.random.default_rng(n * 7 + K)
    keys = rng.integers(0, K, size=n).astype(np.int32)
    perm, rowptr = ba.csr_build(torch.from_numpy(keys).cuda(), K)
    p_ref, r_ref = orc.csr_build(keys, K)
    assert np.array_equal(perm.cpu().numpy(), p_ref)
    assert np.array_equal(rowptr.cpu().numpy(), r_ref)


def test_csr_build_sorted_and_reversed_and_constant():
    n = 50_000
    for keys in (np.arange(n) % 977, np.arange(n)[::-1] // 3, np.full(n, 5)):
        keys = np.ascontiguousarray(keys, dtype=np.int32)
        K = int(keys.max()) + 1
        perm, rowptr = ba.csr_build(torch.from_numpy(keys).cuda(), K)
        p_ref, r_ref = orc.csr_build(keys, K)
        assert np.array_equal(perm.cpu().numpy(), p_ref)
        assert np.array_equal(rowptr.cpu().numpy(), r_ref)


def test_csr_build_rejects_out_of_range():
    keys = torch.tensor([0, 3, 1], dtype=torch.int32, device="cuda")
    with pytest.raises(ba.BAError, match="INVALID_ARG"):
        ba.csr_build(keys, 3)
    keys = torch.tensor([0, -1, 1], dtype=torch.int32, device="cuda")
    with pytest.raises(ba.BAError, match="INVALID_ARG"):
        ba.csr_build(keys, 3)


@pytest.mark.parametrize("which", ["ba16", "ba250"])
def test_problem_csr_bit_exact(which):
    sc = scenegen.config_scene(which, small=True)
    pix = orc.pixels_from_scene(sc)
    with problem(sc, pix) as prob:
        pc, rc, pp, rp = [t.cpu().numpy() for t in prob.csr()]
    p1, r1 = orc.csr_build(sc.cam_idx, sc.C)
    p2, r2 = orc.csr_build(sc.pt_idx, sc.P)
    assert np.array_equal(pc, p1) and np.array_equal(rc, r1)
    assert np.array_equal(pp, p2) and np.array_equal(rp, r2)
