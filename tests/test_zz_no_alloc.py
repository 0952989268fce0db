"""ba_csr_build_noalloc: the allocation-free variant of ba_csr_build, for
callers that may not allocate device memory while running (real-time loops,
processes whose device memory belongs to another allocator).

Called through the C ABI, twice in a row on different sizes (the second call
must not see anything the first left in the shared scratch array), and
compared bit for bit with the oracle's stable counting sort and with
ba_csr_build.  Also checks the entry point's defining property: after a
warm-up call, a full-size call changes the device's free memory by nothing.
Kept in a file collected last, so a run that stops at the first failure has
run every other test before it."""
import ctypes as ct

import numpy as np
import pytest
import torch

import oracle as orc

pytestmark = pytest.mark.gpu


def _abi():
    from paper_2409_12190_gb300 import _lib
    return _lib


def _noalloc_into(keys, n_keys, perm, rowptr):
    _lib = _abi()
    L = _lib.load()
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    kp = ct.c_void_p(keys.data_ptr()) if keys.numel() else None
    pp = ct.c_void_p(perm.data_ptr()) if keys.numel() else None
    _lib.check(L.ba_csr_build_noalloc(kp, keys.shape[0], n_keys, pp, ct.c_void_p(rowptr.data_ptr()),
                                      stream))


def _noalloc(keys, n_keys):
    perm = torch.empty(keys.shape[0], dtype=torch.int32, device="cuda")
    rowptr = torch.empty(n_keys + 1, dtype=torch.int32, device="cuda")
    _noalloc_into(keys, n_keys, perm, rowptr)
    return perm, rowptr


def _existing(keys, n_keys):
    import paper_2409_12190_gb300 as ba
    return ba.csr_build(keys, n_keys)


def _check(keys_np, n_keys, perm, rowptr):
    perm_o, rowptr_o = orc.csr_build(keys_np, n_keys)
    assert np.array_equal(perm.cpu().numpy(), perm_o)
    assert np.array_equal(rowptr.cpu().numpy(), rowptr_o)


def test_noalloc_matches_the_oracle_and_csr_build_on_two_consecutive_calls():
    rng = np.random.default_rng(2024)
    cases = [(300_000, 70_000),   # 3 radix passes, many tiles
             (1_000, 3)]          # small call after a large one: stale scratch must not leak in
    for n, K in cases:
        keys_np = rng.integers(0, K, size=n).astype(np.int32)
        keys = torch.from_numpy(keys_np).cuda()
        perm, rowptr = _noalloc(keys, K)
        torch.cuda.synchronize()
        _check(keys_np, K, perm, rowptr)
        perm_ref, rowptr_ref = _existing(keys, K)
        assert torch.equal(perm, perm_ref) and torch.equal(rowptr, rowptr_ref)


def test_noalloc_allocates_no_device_memory():
    rng = np.random.default_rng(11)
    n_max = 1 << 20
    keys_np = rng.integers(0, 9000, size=n_max).astype(np.int32)
    keys = torch.from_numpy(keys_np).cuda()
    perm = torch.empty(n_max, dtype=torch.int32, device="cuda")
    rowptr = torch.empty(9001, dtype=torch.int32, device="cuda")
    empty = torch.empty(0, dtype=torch.int32, device="cuda")
    _noalloc_into(empty, 1, perm, rowptr)  # warm-up: loads the module and its array
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    _noalloc_into(keys, 9000, perm, rowptr)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    _check(keys_np, 9000, perm, rowptr)


def test_noalloc_at_the_size_limit_and_rejections():
    _lib = _abi()
    import paper_2409_12190_gb300 as ba
    n_max = (1 << 20)
    rng = np.random.default_rng(7)
    keys_np = rng.integers(0, 5000, size=n_max).astype(np.int32)
    keys = torch.from_numpy(keys_np).cuda()
    perm, rowptr = _noalloc(keys, 5000)
    _check(keys_np, 5000, perm, rowptr)
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
