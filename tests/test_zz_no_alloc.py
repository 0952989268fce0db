"""ba_csr_build_noalloc: the allocation-free variant of ba_csr_build, for
callers that may not allocate device memory while running.  Called through
the C ABI and compared with ba_csr_build on the same keys, twice in a row
(the second call must not see anything the first left in the shared
scratch array).  Kept in a file collected last."""
import ctypes as ct

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _abi():
    from paper_2409_12190_gb300 import _lib
    return _lib


def _noalloc(keys, n_keys):
    _lib = _abi()
    L = _lib.load()
    perm = torch.empty(keys.shape[0], dtype=torch.int32, device="cuda")
    rowptr = torch.empty(n_keys + 1, dtype=torch.int32, device="cuda")
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    kp = ct.c_void_p(keys.data_ptr()) if keys.numel() else None
    pp = ct.c_void_p(perm.data_ptr()) if keys.numel() else None
    _lib.check(L.ba_csr_build_noalloc(kp, keys.shape[0], n_keys, pp, ct.c_void_p(rowptr.data_ptr()),
                                      stream))
    return perm, rowptr


def _reference(keys, n_keys):
    import paper_2409_12190_gb300 as ba
    return ba.csr_build(keys, n_keys)


def test_noalloc_matches_csr_build_on_two_consecutive_calls():
    rng = np.random.default_rng(2024)
    cases = [(300_000, 70_000),   # 3 radix passes, many tiles
             (1_000, 3)]          # small call after a large one: stale scratch must not leak in
    for n, K in cases:
        keys = torch.from_numpy(rng.integers(0, K, size=n).astype(np.int32)).cuda()
        perm, rowptr = _noalloc(keys, K)
        perm_ref, rowptr_ref = _reference(keys, K)
        torch.cuda.synchronize()
        assert torch.equal(perm, perm_ref)
        assert torch.equal(rowptr, rowptr_ref)


def test_noalloc_at_the_size_limit_and_rejections():
    _lib = _abi()
    import paper_2409_12190_gb300 as ba
    n_max = (1 << 20)
    rng = np.random.default_rng(7)
    keys = torch.from_numpy(rng.integers(0, 5000, size=n_max).astype(np.int32)).cuda()
    perm, rowptr = _noalloc(keys, 5000)
    perm_ref, rowptr_ref = _reference(keys, 5000)
    assert torch.equal(perm, perm_ref) and torch.equal(rowptr, rowptr_ref)
    # one key more than the fixed maximum is refused before any GPU work
    big = torch.zeros(n_max + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(ba.BAError, match="INVALID_ARG"):
        _noalloc(big, 4)
    assert b"fixed maximum" in _lib.load().ba_last_error()
    # an out-of-range key is reported, and the flag does not stick to the next call
    bad = torch.tensor([0, 9, 1], dtype=torch.int32, device="cuda")
    with pytest.raises(ba.BAError, match="INVALID_ARG"):
        _noalloc(bad, 3)
    good = torch.tensor([2, 0, 1, 0], dtype=torch.int32, device="cuda")
    perm, rowptr = _noalloc(good, 3)
    assert perm.tolist() == [1, 3, 2, 0] and rowptr.tolist() == [0, 2, 3, 4]
