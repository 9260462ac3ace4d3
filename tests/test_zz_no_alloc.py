"""bitsort_noalloc: the sort for callers that cannot allocate device memory.

Some callers of this library cannot call cudaMalloc: applications whose
device memory is all held by another allocator (a caching pool sized to the
whole GPU), and real-time code that forbids allocation after start-up because
an allocation can block for an unbounded time.  bitsort_noalloc keeps its
scratch in a fixed device array of the library instead.  This test calls it
through the C ABI twice in a row and checks that each result is
bit-identical to the CPU oracle's and to the one the allocating entry point
(bitsort_ex) gives for the same keys, and that the calls leave the device's
free memory unchanged.  Collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import gen
import oracle
import paper_1312_0138_gb300 as bs

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _host(t):
    return t.cpu().numpy().view(np.uint32)


def _noalloc(keys, max_value):
    """One call of the C entry point; returns (status, count, output)."""
    import torch
    lib = bs.load()
    out = torch.full_like(keys, -1)
    res = torch.zeros(2, dtype=torch.int64, device="cuda")
    st = lib.bitsort_noalloc(keys.data_ptr(), keys.numel(), max_value, out.data_ptr(), res.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
    assert st == bs.OK, bs.STATUS_NAMES.get(st, st)
    torch.cuda.synchronize()
    r = res.cpu().numpy()
    return int(r[0]) & 0xFFFFFFFF, int(r[1]), _host(out)


def _with_alloc(keys, max_value):
    ctx = bs.default_context()
    st, cnt, out = ctx.sort(keys, max_value)
    return st, cnt, _host(out)


@pytest.mark.parametrize("n,M", [(100_000, 1 << 20), (1 << 22, 1 << 26), (3, 40), (70_001, (1 << 31))])
def test_noalloc_matches_oracle_and_allocating_entry_point_twice(n, M):
    keys_np = gen.floyd(4242 + n, n, M)
    keys = _dev(keys_np)
    oracle_st, oracle_out = oracle.bitmap_sort(keys_np, M - 1)
    want_st, want_cnt, want = _with_alloc(keys, M - 1)
    assert want_st == oracle_st == bs.OK
    assert np.array_equal(want[:want_cnt], oracle_out)
    for _ in range(2):   # the shared scratch keeps the last call's contents
        st, cnt, got = _noalloc(keys, M - 1)
        assert (st, cnt) == (oracle_st, oracle_out.size) == (want_st, want_cnt)
        assert np.array_equal(got[:cnt], oracle_out)
        assert np.array_equal(got[:cnt], want[:want_cnt])


def test_noalloc_error_semantics_match():
    # duplicates and keys above max_value give the oracle's outcome, and the
    # allocating entry point's, both ways
    for keys_np, mv in [(gen.uniform_with_replacement(7, 50_000, 1 << 16), (1 << 16) - 1),
                        (gen.floyd(8, 30_000, 1 << 20), (1 << 19) + 5)]:
        keys = _dev(keys_np)
        want = _with_alloc(keys, mv)
        o_st, o_out = oracle.bitmap_sort(keys_np, mv)
        assert want[:2] == (o_st, o_out.size)
        for _ in range(2):
            got = _noalloc(keys, mv)
            assert got[:2] == want[:2]
            assert np.array_equal(got[2][: got[1]], o_out)
            assert np.array_equal(got[2][: got[1]], want[2][: want[1]])


def test_noalloc_leaves_free_device_memory_unchanged():
    import torch
    keys_np = gen.floyd(99, 1 << 20, 1 << 26)
    keys = _dev(keys_np)
    out = torch.empty_like(keys)
    res = torch.zeros(2, dtype=torch.int64, device="cuda")
    lib = bs.load()
    s = torch.cuda.current_stream().cuda_stream
    assert lib.bitsort_noalloc(keys.data_ptr(), keys.numel(), (1 << 26) - 1, out.data_ptr(), res.data_ptr(), s) == bs.OK
    torch.cuda.synchronize()   # the first call on a device finds its scratch array
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert lib.bitsort_noalloc(keys.data_ptr(), keys.numel(), (1 << 26) - 1, out.data_ptr(), res.data_ptr(),
                                   s) == bs.OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    r = res.cpu().numpy()
    assert int(r[0]) & 0xFFFFFFFF == bs.OK and int(r[1]) == keys_np.size
    assert np.array_equal(_host(out), np.sort(keys_np))


def test_noalloc_rejects_what_it_cannot_hold():
    import torch
    lib = bs.load()
    keys = _dev(np.arange(10, dtype=np.uint32))
    res = torch.zeros(2, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    # in place: the output buffer is the partition buffer
    assert lib.bitsort_noalloc(keys.data_ptr(), 10, 100, keys.data_ptr(), res.data_ptr(), s) == bs.ERR_INVALID
    # a range beyond the fixed scratch (max_value >= 2^31)
    out = torch.empty_like(keys)
    assert lib.bitsort_noalloc(keys.data_ptr(), 10, 1 << 31, out.data_ptr(), res.data_ptr(), s) == bs.ERR_INVALID
    # no place for the outcome
    assert lib.bitsort_noalloc(keys.data_ptr(), 10, 100, out.data_ptr(), None, s) == bs.ERR_INVALID
