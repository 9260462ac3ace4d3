"""Parity of the signed sort (bitsort_i32: int32 keys in [min_value,
max_value], Algorithm 1's second function) with the CPU oracle, through the
C ABI, on every path."""
import numpy as np
import pytest

import gen
import oracle
import paper_1312_0138_gb300 as bs

pytestmark = pytest.mark.gpu

I32MIN, I32MAX = -(1 << 31), (1 << 31) - 1


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    bs.load()
    c = bs.Context(0)
    yield c
    c.close()


def signed_keys(seed, n, lo, hi):
    """n distinct int32 keys in [lo, hi]: distinct offsets in [0, hi - lo]
    moved to start at lo (two's complement wrap)."""
    span = hi - lo + 1
    off = gen.keys(seed, n, span).astype(np.uint64)
    return ((off + np.uint64(lo & 0xFFFFFFFF)) & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.int32)


def gpu_sort_i32(ctx, keys, lo, hi, inplace=False, path=None, S=0, threads=0, **cfg):
    import torch
    n = keys.size
    if path is not None:   # the configuration is looked up by the span of the range
        ctx.set_config(max(n, 1), hi - lo, path, S, threads, **cfg)
    d = torch.from_numpy(np.ascontiguousarray(keys, dtype=np.int32)).cuda()
    out = d if inplace else torch.empty_like(d)
    try:
        st, cnt, out = ctx.sort_i32(d, lo, hi, out=out)
    finally:
        if path is not None:
            ctx.set_config(max(n, 1), hi - lo, bs.PATH_AUTO)
    assert st != bs.ERR_TIMEOUT
    return st, cnt, out.cpu().numpy()[:cnt]


def check(ctx, keys, lo, hi, **kw):
    want_st, want = oracle.default().bitmap_sort_i32(keys, lo, hi)
    st, cnt, got = gpu_sort_i32(ctx, keys, lo, hi, **kw)
    assert st == want_st, (st, want_st, kw)
    assert cnt == want.size
    assert np.array_equal(got, want), kw
    return got


RANGES = [
    ("full_int32", I32MIN, I32MAX, 300_001),
    ("straddles_zero", -1_000_003, 3_000_017, 250_000),
    ("negative_only", I32MIN, -(1 << 30), 120_000),
    ("nonnegative_top", (1 << 30), I32MAX, 90_001),
    ("tiny_negative", -40, -3, 30),
    ("small_straddle_fused", -5000, 5000, 7000),
]
PATHS = [
    ("auto", None, 0, 0, {}),
    ("fused", bs.PATH_FUSED, 0, 512, {}),
    ("exact_S4096", bs.PATH_PARTITION, 4096, 256, dict(layout=0)),
    ("cap_S64K", bs.PATH_PARTITION, 1 << 16, 512, dict(layout=1)),
    ("exact_persist", bs.PATH_PARTITION, 300_032, 512, dict(layout=0, persistent=1)),
    ("rank_cap", bs.PATH_PARTITION, 1 << 16, 512, dict(layout=1, emit=1)),
    ("global_S64K", bs.PATH_GLOBAL, 1 << 16, 512, {}),
    ("stream_part", bs.PATH_PARTITION, 1 << 16, 512, dict(layout=1, part_stream=1)),
]


@pytest.mark.parametrize("name,lo,hi,n", RANGES, ids=[r[0] for r in RANGES])
@pytest.mark.parametrize("pname,path,S,T,cfg", PATHS, ids=[p[0] for p in PATHS])
def test_signed_parity(ctx, name, lo, hi, n, pname, path, S, T, cfg):
    if path == bs.PATH_FUSED and hi - lo + 1 > (1 << 20):
        pytest.skip("one slice holds at most 2^20 values")
    keys = signed_keys(gen.SEED_BASE + 71 + n, n, lo, hi)
    got = check(ctx, keys, lo, hi, path=path, S=S, threads=T, **cfg)
    # the signed order itself, and Algorithm 1 with its sign split agree
    assert np.array_equal(got, np.sort(keys))
    if n <= 10_000:
        assert np.array_equal(got, oracle.paper_sort_i32(keys))


def test_signed_extremes_and_in_place(ctx):
    keys = np.array([I32MAX, 0, I32MIN, -1, 1, I32MIN + 1, I32MAX - 1], np.int32)
    got = check(ctx, keys, I32MIN, I32MAX, inplace=True)
    assert got.tolist() == sorted(keys.tolist())


def test_signed_single_value_range(ctx):
    for v in (I32MIN, -7, 0, I32MAX):
        check(ctx, np.array([v], np.int32), v, v)


def test_signed_key_range_errors(ctx):
    lo, hi = -1000, 1000
    base = signed_keys(gen.SEED_BASE + 5, 500, lo, hi)
    for bad in (lo - 1, hi + 1, I32MIN, I32MAX):
        keys = base.copy()
        keys[123] = bad
        want_st, _ = oracle.default().bitmap_sort_i32(keys, lo, hi)
        assert want_st == bs.ERR_KEY_RANGE
        st, _, _ = gpu_sort_i32(ctx, keys, lo, hi)
        assert st == bs.ERR_KEY_RANGE, bad


def test_signed_duplicates(ctx):
    lo, hi = -(1 << 24), (1 << 24)
    keys = signed_keys(gen.SEED_BASE + 6, 200_000, lo, hi)
    keys[77_777] = keys[3]
    want_st, _ = oracle.default().bitmap_sort_i32(keys, lo, hi)
    assert want_st == bs.ERR_DUPLICATE
    st, _, _ = gpu_sort_i32(ctx, keys, lo, hi)
    assert st == bs.ERR_DUPLICATE


def test_signed_host_errors(ctx):
    import torch
    d = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(bs.BitsortError) as e:
        ctx.sort_i32_async(d, 5, 4)   # min_value > max_value
    assert e.value.status == bs.ERR_INVALID
    with pytest.raises(bs.BitsortError) as e:
        ctx.sort_i32_async(d, -1, 1)  # four keys cannot be distinct in three values
    assert e.value.status == bs.ERR_INVALID
    st, cnt, _ = ctx.sort_i32(d[:0], -3, 3)
    assert st == bs.OK and cnt == 0


def test_signed_default_context_entry(ctx):
    import torch
    keys = signed_keys(gen.SEED_BASE + 9, 50_000, -(1 << 20), 1 << 20)
    d = torch.from_numpy(keys).cuda()
    out = bs.bitsort_i32(d, -(1 << 20), 1 << 20)
    st, cnt = bs.default_context(0).sync_status()
    assert st == bs.OK and cnt == keys.size
    assert np.array_equal(out.cpu().numpy(), np.sort(keys))


@pytest.mark.parametrize("layout", [0, 1])
def test_wide_partition_signed_bias(ctx, layout):
    # the partition classifies x - min_value: signed keys straddling zero,
    # 2048 buckets (the partition at 1024 threads, buckets by shift)
    lo, hi = -(1 << 24), (1 << 24) - 1
    keys = signed_keys(64, 1 << 23, lo, hi)
    check(ctx, keys, lo, hi, path=bs.PATH_PARTITION, S=1 << 14, threads=512, layout=layout)
