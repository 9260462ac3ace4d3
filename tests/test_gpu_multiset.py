"""Parity of the multiset path (bitsort_multiset: Algorithm 1's stable bit
splits on the GPU, keys may repeat) with the CPU oracle's Algorithm 1,
through the C ABI: every split width, repeated and distinct keys, ragged
tiles, in place, signed keys, range errors."""
import numpy as np
import pytest

import gen
import oracle
import paper_1312_0138_gb300 as bs

pytestmark = pytest.mark.gpu

TILE = 4096
I32MIN, I32MAX = -(1 << 31), (1 << 31) - 1


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    bs.load()
    c = bs.Context(0)
    yield c
    c.close()


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def gpu_multiset(ctx, keys, max_value, split_bits=0, inplace=False, offset=0):
    import torch
    n = keys.size
    if offset:   # keys and out start `offset` elements into their allocations
        kb = dev(np.concatenate([np.zeros(offset, np.uint32), keys]))
        d = kb[offset:]
        ob = torch.empty(n + offset, dtype=torch.int32, device="cuda")
        out = ob[offset:]
    else:
        d = dev(keys)
        out = d if inplace else torch.empty_like(d)
    st, cnt, out = ctx.multiset(d, max_value, split_bits, out=out)
    assert st != bs.ERR_TIMEOUT
    return st, cnt, out.cpu().numpy().view(np.uint32)


def check(ctx, keys, max_value, split_bits=0, **kw):
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    want = oracle.paper_sort_u32(keys)            # Algorithm 1 on the CPU, all 32 bits
    st, cnt, got = gpu_multiset(ctx, keys, max_value, split_bits, **kw)
    assert st == bs.OK, st
    assert cnt == keys.size
    assert np.array_equal(got, want), (split_bits, kw)
    return got


def bits_of(max_value):
    return max(1, int(max_value).bit_length())


CASES = [
    # (name, n, max_value, generator)
    ("distinct_c0", 100_000, (1 << 20) - 1, "distinct"),
    ("repeats_small_range", 70_001, 999, "repeat"),
    ("repeats_wide", 123_457, (1 << 32) - 1, "repeat"),
    ("all_equal", 9_000, 12345, "equal"),
    ("one_tile_ragged", TILE - 3, (1 << 16) - 1, "repeat"),
    ("many_tiles_ragged", 37 * TILE + 1, (1 << 24) - 1, "repeat"),
    ("max_value_zero", 5_000, 0, "zeros"),
]


def make(kind, seed, n, max_value):
    M = max_value + 1
    if kind == "distinct":
        return gen.keys(seed, n, M)
    if kind == "repeat":
        return gen.uniform_with_replacement(seed, n, M)
    if kind == "equal":
        return np.full(n, max_value // 3, np.uint32)
    return np.zeros(n, np.uint32)


@pytest.mark.parametrize("split_bits", [0, 1, 3, 4, 7, 8])
@pytest.mark.parametrize("name,n,max_value,kind", CASES, ids=[c[0] for c in CASES])
def test_multiset_parity(ctx, name, n, max_value, kind, split_bits):
    keys = make(kind, gen.SEED_BASE + 300 + n, n, max_value)
    got = check(ctx, keys, max_value, split_bits)
    assert np.array_equal(got, np.sort(keys))


@pytest.mark.parametrize("split_bits", [2, 5, 6])
def test_multiset_other_widths(ctx, split_bits):
    keys = gen.uniform_with_replacement(gen.SEED_BASE + 41, 50_000, 1 << 28)
    check(ctx, keys, (1 << 28) - 1, split_bits)


def test_multiset_distinct_equals_bitmap_path(ctx):
    # on distinct keys the two forms of the paper's sort give the same array
    n, M = 300_000, 1 << 24
    keys = gen.keys(gen.SEED_BASE + 42, n, M)
    got = check(ctx, keys, M - 1)
    st, want = oracle.bitmap_sort(keys, M - 1)
    assert st == bs.OK and np.array_equal(got, want)


@pytest.mark.parametrize("max_value,split_bits", [((1 << 20) - 1, 0), ((1 << 20) - 1, 4), ((1 << 21) - 1, 7),
                                                  (255, 8), (255, 0)])
def test_multiset_in_place(ctx, max_value, split_bits):
    # odd and even numbers of passes, including one pass
    keys = gen.uniform_with_replacement(gen.SEED_BASE + 43 + split_bits, 77_777, max_value + 1)
    check(ctx, keys, max_value, split_bits, inplace=True)


def test_multiset_unaligned(ctx):
    keys = gen.uniform_with_replacement(gen.SEED_BASE + 44, 20_003, 1 << 20)
    check(ctx, keys, (1 << 20) - 1, 0, offset=1)
    check(ctx, keys, (1 << 20) - 1, 0, offset=3)


def test_multiset_tiny(ctx):
    for n in (1, 2, 31, 32, 33):
        keys = gen.uniform_with_replacement(gen.SEED_BASE + 45 + n, n, 10)
        check(ctx, keys, 9, 0)
        check(ctx, keys, 9, 1)


def test_multiset_empty(ctx):
    import torch
    d = torch.empty(0, dtype=torch.int32, device="cuda")
    st, cnt, _ = ctx.multiset(d, 100)
    assert st == bs.OK and cnt == 0


def test_multiset_key_range(ctx):
    keys = gen.uniform_with_replacement(gen.SEED_BASE + 46, 50_000, 1000)
    keys[777] = 1000   # one above max_value = 999
    st, cnt, got = gpu_multiset(ctx, keys, 999)
    assert st == bs.ERR_KEY_RANGE and cnt == keys.size
    # the context serves the next call normally
    check(ctx, keys[:777], 999)


def test_multiset_host_errors(ctx):
    import torch
    d = torch.zeros(100, dtype=torch.int32, device="cuda")
    with pytest.raises(bs.BitsortError) as e:
        ctx.multiset_async(d, 100, split_bits=9)
    assert e.value.status == bs.ERR_INVALID
    with pytest.raises(bs.BitsortError) as e:
        ctx.multiset_async(d[:60], 100, out=d[40:])   # partial overlap
    assert e.value.status == bs.ERR_INVALID


SIGNED = [
    ("full", I32MIN, I32MAX, 200_001),
    ("straddle", -5000, 5000, 90_000),
    ("negative", I32MIN, -(1 << 20), 30_000),
]


@pytest.mark.parametrize("split_bits", [0, 1, 8])
@pytest.mark.parametrize("name,lo,hi,n", SIGNED, ids=[s[0] for s in SIGNED])
def test_multiset_signed(ctx, name, lo, hi, n, split_bits):
    import torch
    span = hi - lo + 1
    off = gen.uniform_with_replacement(gen.SEED_BASE + 47 + n, n, span).astype(np.uint64)
    keys = ((off + np.uint64(lo & 0xFFFFFFFF)) & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.int32)
    want = oracle.paper_sort_i32(keys)   # Algorithm 1 with its sign split
    d = torch.from_numpy(keys.copy()).cuda()
    st, cnt, out = ctx.multiset_i32(d, lo, hi, split_bits)
    assert st == bs.OK and cnt == n
    got = out.cpu().numpy()
    assert np.array_equal(got, want)
    assert np.array_equal(got, np.sort(keys))


def test_multiset_signed_range_error(ctx):
    import torch
    keys = np.array([-3, 5, 2, -3, 7], np.int32)
    st, _, _ = ctx.multiset_i32(torch.from_numpy(keys).cuda(), -3, 6)
    assert st == bs.ERR_KEY_RANGE
    with pytest.raises(bs.BitsortError):
        ctx.multiset_i32_async(torch.from_numpy(keys).cuda(), 1, 0)


def test_multiset_phase_timing(ctx):
    import torch
    keys = gen.uniform_with_replacement(gen.SEED_BASE + 48, 1 << 20, 1 << 28)
    d = dev(keys)
    ctx.set_phase_timing(True)
    try:
        st, cnt, out = ctx.multiset(d, (1 << 28) - 1)
        times = ctx.phase_times()
    finally:
        ctx.set_phase_timing(False)
    assert st == bs.OK
    assert [k for k, _ in times] == ["mhist", "msplit"]
    assert all(ms > 0 for _, ms in times)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), np.sort(keys))
