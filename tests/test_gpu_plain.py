"""Parity of the GPU bitmap sort with the CPU oracle (bit-exact), single
arrays, every path and slice size, through the C ABI."""
import numpy as np
import pytest

import gen
import oracle
import paper_1312_0138_gb300 as bs
from gpu_util import gpu_sort, to_dev, to_host

pytestmark = pytest.mark.gpu

U32MAX = (1 << 32) - 1


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    bs.load()
    c = bs.Context(0)
    yield c
    c.close()


def check(ctx, keys, max_value, **kw):
    want_st, want = oracle.bitmap_sort(keys, max_value)
    st, cnt, got = gpu_sort(ctx, keys, max_value, **kw)
    assert st == want_st, (st, want_st, kw)
    assert cnt == want.size, (cnt, want.size, kw)
    assert np.array_equal(got, want), kw


# sizes span several tiles (8192 / 4096 keys) with ragged tails, slices with
# partial last words, and values up to 2^32 - 1
SIZES = [(1, 1), (3, 40), (1000, 1 << 12), (4097, 8200), (40_000, 300_007),
         (100_000, 1 << 20), (70_001, 1 << 24), (20_000, 1 << 32), (262_147, 1 << 19)]
CONFIGS = [
    ("fused512", bs.PATH_FUSED, 0, 512),
    ("fused256", bs.PATH_FUSED, 0, 256),
    ("part_S128", bs.PATH_PARTITION, 128, 512),
    ("part_S4096_256", bs.PATH_PARTITION, 4096, 256),
    ("part_S65536", bs.PATH_PARTITION, 1 << 16, 512),
    ("part_S1M", bs.PATH_PARTITION, 1 << 20, 512),
    ("part_odd", bs.PATH_PARTITION, 883_072, 512),
    ("global_S16K", bs.PATH_GLOBAL, 1 << 14, 512),
    ("global_S1M_256", bs.PATH_GLOBAL, 1 << 20, 256),
]


@pytest.mark.parametrize("name,path,S,threads", CONFIGS, ids=[c[0] for c in CONFIGS])
@pytest.mark.parametrize("n,M", SIZES, ids=[f"n{n}_M{M}" for n, M in SIZES])
def test_parity_paths(ctx, name, path, S, threads, n, M):
    if path == bs.PATH_FUSED and M > (1 << 20):
        pytest.skip("fused needs the whole bitmap in one CTA")
    keys = gen.floyd(hash((n, M)) & 0xFFFF, n, M)
    check(ctx, keys, M - 1, path=path, S=S, threads=threads)


def test_config0_default_path(ctx):
    keys = gen.floyd(gen.SEED_BASE + 0, 100_000, 1 << 20)
    check(ctx, keys, (1 << 20) - 1)


def test_full_permutation_closed_form(ctx):
    for M in (32, 1000, 1 << 16, (1 << 20) + 5):
        keys = gen.feistel(M, M, M)
        st, cnt, got = gpu_sort(ctx, keys, M - 1)
        assert st == bs.OK and np.array_equal(got, np.arange(M, dtype=np.uint32))


def test_empty_and_single(ctx):
    import torch
    st, cnt, out = ctx.sort(torch.empty(0, dtype=torch.int32, device="cuda"), 10)
    assert st == bs.OK and cnt == 0
    check(ctx, np.array([0], np.uint32), 0)
    check(ctx, np.array([7], np.uint32), 7)
    check(ctx, np.array([U32MAX], np.uint32), U32MAX)


def test_extremes_full_range(ctx):
    keys = np.array([U32MAX, 0, 1 << 31, (1 << 31) - 1, U32MAX - 1, 12345], np.uint32)
    for path in (None, bs.PATH_PARTITION, bs.PATH_GLOBAL):
        check(ctx, keys, U32MAX, path=path)


@pytest.mark.parametrize("path", [bs.PATH_FUSED, bs.PATH_PARTITION, bs.PATH_GLOBAL])
def test_in_place(ctx, path):
    keys = gen.floyd(77, 50_000, 1 << 20)
    check(ctx, keys, (1 << 20) - 1, path=path, inplace=True)


@pytest.mark.parametrize("path", [bs.PATH_FUSED, bs.PATH_PARTITION, bs.PATH_GLOBAL])
@pytest.mark.parametrize("offset", [1, 2, 3])
def test_unaligned_pointers(ctx, path, offset):
    keys = gen.floyd(78 + offset, 33_333, 1 << 20)
    check(ctx, keys, (1 << 20) - 1, path=path, offset=offset)


@pytest.mark.parametrize("path", [bs.PATH_FUSED, bs.PATH_PARTITION, bs.PATH_GLOBAL])
def test_duplicates_give_distinct_prefix(ctx, path):
    keys = gen.uniform_with_replacement(5, 60_000, 1 << 16)
    check(ctx, keys, (1 << 16) - 1, path=path)
    keys = np.array([3, 3, 3, 3], np.uint32)
    check(ctx, keys, 3, path=path)


@pytest.mark.parametrize("path", [bs.PATH_FUSED, bs.PATH_PARTITION, bs.PATH_GLOBAL])
def test_key_range_skips_and_reports(ctx, path):
    keys = gen.floyd(9, 20_000, 1 << 18)
    mv = (1 << 17) + 3   # about half the keys are out of range
    check(ctx, keys, mv, path=path)


def test_host_errors(ctx):
    import torch
    keys = to_dev(np.arange(10, dtype=np.uint32))
    with pytest.raises(bs.BitsortError) as e:
        ctx.sort_async(keys, 5)          # n > max_value + 1: cannot be distinct
    assert e.value.status == bs.ERR_INVALID
    buf = torch.zeros(20, dtype=torch.int32, device="cuda")
    with pytest.raises(bs.BitsortError):
        ctx.sort_async(buf[:10], 100, out=buf[5:15])   # partial overlap


def test_plain_entry_point_default_context():
    keys_np = gen.floyd(11, 5000, 1 << 20)
    keys = to_dev(keys_np)
    out = bs.bitsort(keys, (1 << 20) - 1)
    st, cnt = bs.sync_status()
    assert st == bs.OK and cnt == keys_np.size
    assert np.array_equal(to_host(out), np.sort(keys_np))


def test_device_result_pointer(ctx):
    import torch
    keys_np = gen.floyd(12, 4000, 1 << 14)
    res = torch.zeros(2, dtype=torch.int64, device="cuda")
    out = ctx.sort_async(to_dev(keys_np), (1 << 14) - 1, result=res)
    torch.cuda.synchronize()
    r = res.cpu().numpy()
    assert int(r[0]) & 0xFFFFFFFF == bs.OK and int(r[1]) == keys_np.size
    assert np.array_equal(to_host(out), np.sort(keys_np))


def test_repeated_calls_keep_scratch_clean(ctx):
    # the scratch is returned to zero by the kernel itself: many calls in a
    # row, alternating paths and sizes, stay exact
    for i in range(12):
        n, M = [(5000, 1 << 16), (70_000, 1 << 22), (3, 1 << 32)][i % 3]
        path = [bs.PATH_PARTITION, bs.PATH_GLOBAL, None][i % 3]
        check(ctx, gen.floyd(100 + i, n, M), M - 1, path=path)


def test_autotune_picks_a_correct_config(ctx, tmp_path):
    import torch
    keys_np = gen.floyd(13, 1 << 18, 1 << 22)
    keys = to_dev(keys_np)
    best = ctx.autotune(keys, (1 << 22) - 1, out=torch.empty_like(keys))
    assert best["path"] in ("fused", "partition", "global") and best["ms"] > 0
    assert ctx.get_config(1 << 18, (1 << 22) - 1)["path"] == best["path"]
    check(ctx, keys_np, (1 << 22) - 1)
    p = str(tmp_path / "tune.json")
    ctx.tune_save(p)
    c2 = bs.Context(0)
    c2.tune_load(p)
    assert c2.get_config(1 << 18, (1 << 22) - 1) == ctx.get_config(1 << 18, (1 << 22) - 1)
    c2.close()
