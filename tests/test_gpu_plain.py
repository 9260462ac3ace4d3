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
    ("fused512_w1_stage", bs.PATH_FUSED, 0, 512, dict(words_per_lane=1, stage=1)),
    ("fused256_w4", bs.PATH_FUSED, 0, 256, dict(words_per_lane=4)),
    ("fused512_w2_persist", bs.PATH_FUSED, 0, 512, dict(words_per_lane=2, persistent=1)),
    ("exact_S128_w1", bs.PATH_PARTITION, 128, 512, dict(layout=0, words_per_lane=1)),
    ("cap_S4096_256_w2", bs.PATH_PARTITION, 4096, 256, dict(layout=1, words_per_lane=2)),
    ("exact_S64K_stage", bs.PATH_PARTITION, 1 << 16, 512, dict(layout=0, stage=1)),
    ("cap_S1M_w4", bs.PATH_PARTITION, 1 << 20, 512, dict(layout=1, words_per_lane=4)),
    ("cap_odd_persist", bs.PATH_PARTITION, 883_072, 256, dict(layout=1, persistent=1, words_per_lane=2)),
    ("exact_odd_persist_stage", bs.PATH_PARTITION, 883_072, 512, dict(layout=0, persistent=1, stage=1)),
    ("exact_S4096_persist_w4", bs.PATH_PARTITION, 4096, 256, dict(layout=0, persistent=1, words_per_lane=4)),
    ("cap_S1M_runs8", bs.PATH_PARTITION, 1 << 20, 512, dict(layout=1, stage=1, words_per_lane=8)),
    ("cap_stream_S64K", bs.PATH_PARTITION, 1 << 16, 512, dict(layout=1, part_stream=1)),
    ("exact_stream_odd_256", bs.PATH_PARTITION, 300_032, 256, dict(layout=0, part_stream=1)),
    # 1024 or more buckets: the streaming partition runs at 1024 threads (16 Ki-key tiles)
    ("cap_stream_S4096_wide", bs.PATH_PARTITION, 4096, 512, dict(layout=1, part_stream=1)),
    ("exact_stream_S16K_wide", bs.PATH_PARTITION, 16384, 512, dict(layout=0, part_stream=1)),
    ("exact_odd_runs4_256", bs.PATH_PARTITION, 300_032, 256, dict(layout=0, stage=1, words_per_lane=4)),
    ("cap_S4096_runs8_persist", bs.PATH_PARTITION, 4096, 512, dict(layout=1, stage=1, words_per_lane=8,
                                                                    persistent=1)),
    ("fused_runs8", bs.PATH_FUSED, 0, 512, dict(stage=1, words_per_lane=8)),
    ("global_S64K_runs4", bs.PATH_GLOBAL, 1 << 16, 512, dict(stage=1, words_per_lane=4)),
    ("rank_cap_S64K", bs.PATH_PARTITION, 1 << 16, 512, dict(layout=1, emit=1)),
    ("rank_exact_S4096_256", bs.PATH_PARTITION, 4096, 256, dict(layout=0, emit=1)),
    ("rank_exact_odd_persist", bs.PATH_PARTITION, 300_032, 512, dict(layout=0, emit=1, persistent=1)),
    ("rank_cap_S1M_persist", bs.PATH_PARTITION, 1 << 20, 256, dict(layout=1, emit=1, persistent=1)),
    ("fused1024", bs.PATH_FUSED, 0, 1024, dict(words_per_lane=1)),
    ("exact_S4096_1024", bs.PATH_PARTITION, 4096, 1024, dict(layout=0)),
    ("cap_S64K_1024_w2", bs.PATH_PARTITION, 1 << 16, 1024, dict(layout=1, words_per_lane=2)),
    ("global_S64K_1024", bs.PATH_GLOBAL, 1 << 16, 1024, {}),
    ("exact_S1M_1024_stage", bs.PATH_PARTITION, 1 << 20, 1024, dict(layout=0, stage=1)),
    ("rank_fused", bs.PATH_FUSED, 0, 512, dict(emit=1)),
    ("global_S16K_w1", bs.PATH_GLOBAL, 1 << 14, 512, dict(words_per_lane=1)),
    ("global_S1M_256_w4", bs.PATH_GLOBAL, 1 << 20, 256, dict(words_per_lane=4)),
    ("global_S64K_persist_stage", bs.PATH_GLOBAL, 1 << 16, 256, dict(persistent=1, stage=1)),
    # partition tiles with a power-of-two slice (bucket by shift) and with any slice
    ("cap_S4096_pow2", bs.PATH_PARTITION, 4096, 512, dict(layout=1)),
    ("exact_S1M_w2_pow2", bs.PATH_PARTITION, 1 << 20, 512, dict(layout=0, words_per_lane=2)),
    ("cap_odd_256", bs.PATH_PARTITION, 300_032, 256, dict(layout=1)),
    ("cap_odd_1024", bs.PATH_PARTITION, 883_072, 1024, dict(layout=1)),
    # the partition phase at a block size of its own
    ("cap_S4096_part512", bs.PATH_PARTITION, 4096, 512, dict(layout=1, part_threads=512)),
    ("exact_S4096_part256", bs.PATH_PARTITION, 4096, 512, dict(layout=0, part_threads=256)),
    ("cap_S64K_part1024_stage", bs.PATH_PARTITION, 1 << 16, 512, dict(layout=1, part_threads=1024, stage=1)),
    # wide partition tiles (32 Ki keys at 1024 threads): one tile per CTA at these sizes
    ("cap_S4096_wide", bs.PATH_PARTITION, 4096, 512, dict(layout=1, part_threads=1024, part_tile_keys=32768)),
    ("exact_odd_wide", bs.PATH_PARTITION, 300_032, 512, dict(layout=0, part_threads=1024, part_tile_keys=32768)),
    ("cap_odd_wide512", bs.PATH_PARTITION, 883_072, 512, dict(layout=1, part_threads=512, part_tile_keys=16384)),
    ("exact_S4096_wide512", bs.PATH_PARTITION, 4096, 512, dict(layout=0, part_threads=512, part_tile_keys=16384)),
]


@pytest.mark.parametrize("name,path,S,threads,extra", CONFIGS, ids=[c[0] for c in CONFIGS])
@pytest.mark.parametrize("n,M", SIZES, ids=[f"n{n}_M{M}" for n, M in SIZES])
def test_parity_paths(ctx, name, path, S, threads, extra, n, M):
    if path == bs.PATH_FUSED and M > (1 << 20):
        pytest.skip("fused needs the whole bitmap in one CTA")
    keys = gen.floyd(hash((n, M)) & 0xFFFF, n, M)
    check(ctx, keys, M - 1, path=path, S=S, threads=threads, **extra)


# the four strategies the error-path tests run through
STRATS = [
    ("fused", dict(path=bs.PATH_FUSED)),
    ("exact", dict(path=bs.PATH_PARTITION, S=4096, layout=0)),
    ("capacity", dict(path=bs.PATH_PARTITION, S=4096, layout=1)),
    ("global", dict(path=bs.PATH_GLOBAL, S=4096)),
    ("rank_exact", dict(path=bs.PATH_PARTITION, S=4096, layout=0, emit=1)),
    ("rank_capacity", dict(path=bs.PATH_PARTITION, S=4096, layout=1, emit=1)),
    ("rank_fused", dict(path=bs.PATH_FUSED, emit=1)),
    ("runs8", dict(path=bs.PATH_PARTITION, S=4096, layout=1, stage=1, words_per_lane=8)),
    ("stream", dict(path=bs.PATH_PARTITION, S=4096, layout=1, part_stream=1)),
]


@pytest.mark.parametrize("layout", [0, 1])
def test_stream_partition_many_tiles_per_cta(ctx, layout):
    # 4096 buckets: the streaming partition runs at 1024 threads, one CTA per
    # SM, so each CTA takes several 16 Ki-key tiles through both landing
    # buffers; the odd n leaves a ragged last tile loaded by the threads
    keys = gen.floyd(gen.SEED_BASE + 77, 8_000_009, 1 << 24)
    check(ctx, keys, (1 << 24) - 1, path=bs.PATH_PARTITION, S=4096, threads=512, layout=layout, part_stream=1)


@pytest.mark.parametrize("layout", [0, 1])
def test_rank_emission_falls_back_on_skewed_slices(ctx, layout):
    # every key in the first slice: far more outputs than the staging room
    # planned from the average density, so that slice walks its words
    keys = gen.floyd(31, 4000, 4096)
    check(ctx, keys, (1 << 20) - 1, path=bs.PATH_PARTITION, S=4096, layout=layout, emit=1)
    keys = np.concatenate([gen.floyd(32, 3000, 4096), (gen.floyd(33, 3000, (1 << 20) - 13) + 4096).astype(np.uint32)])
    keys = np.unique(keys)
    check(ctx, gen.shuffle(34, keys), (1 << 20) + 4096, path=bs.PATH_PARTITION, S=4096, layout=layout, emit=1)


def test_default_plan_n100k_range_2e20(ctx):
    keys = gen.floyd(gen.SEED_BASE + 0, 100_000, 1 << 20)
    check(ctx, keys, (1 << 20) - 1)


def test_default_layout_by_scratch():
    # the capacity layout's buffer (about 4 bytes per value of the range) is
    # allowed up to 4 GiB, or up to twice the keys' own bytes: dense 2^31
    # keys over 2^32 values use it, sparse 2^24 keys over 2^32 values take
    # the exact layout (no buffer beyond the output)
    c = bs.Context(0)
    try:
        assert c.get_config(1 << 31, (1 << 32) - 1)["layout"] == "capacity"
        assert c.get_config(1 << 24, (1 << 32) - 1)["layout"] == "exact"
        assert c.get_config(1 << 24, (1 << 28) - 1)["layout"] == "capacity"
    finally:
        c.close()


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
    for strat in [dict()] + [st for name, st in STRATS if name != "fused"]:
        check(ctx, keys, U32MAX, **strat)


@pytest.mark.parametrize("name,strat", STRATS, ids=[x[0] for x in STRATS])
def test_in_place(ctx, name, strat):
    keys = gen.floyd(77, 50_000, 1 << 20)
    check(ctx, keys, (1 << 20) - 1, inplace=True, **strat)


@pytest.mark.parametrize("name,strat", STRATS, ids=[x[0] for x in STRATS])
@pytest.mark.parametrize("offset", [1, 2, 3])
def test_unaligned_pointers(ctx, name, strat, offset):
    keys = gen.floyd(78 + offset, 33_333, 1 << 20)
    check(ctx, keys, (1 << 20) - 1, offset=offset, **strat)


@pytest.mark.parametrize("name,strat", STRATS, ids=[x[0] for x in STRATS])
def test_duplicates_give_distinct_prefix(ctx, name, strat):
    keys = gen.uniform_with_replacement(5, 60_000, 1 << 16)
    check(ctx, keys, (1 << 16) - 1, **strat)
    keys = np.array([3, 3, 3, 3], np.uint32)
    check(ctx, keys, 3, **strat)


@pytest.mark.parametrize("layout,persistent", [(1, 0), (1, 1)])
def test_capacity_overflow_from_repeated_keys(ctx, layout, persistent):
    # one bucket receives more keys than it can hold (only possible with
    # repeats): that bucket is rebuilt from the whole input
    rep = np.full(30_000, 5, np.uint32)
    rest = gen.floyd(21, 20_000, 1 << 18)
    keys = gen.shuffle(22, np.concatenate([rep, rest]))
    check(ctx, keys, (1 << 18) - 1, path=bs.PATH_PARTITION, S=4096, layout=layout, persistent=persistent)
    check(ctx, keys, (1 << 18) - 1, path=bs.PATH_PARTITION, S=4096, layout=layout, persistent=persistent,
          inplace=True)


@pytest.mark.parametrize("order", ["random", "ascending", "descending", "runs"])
@pytest.mark.parametrize("S,layout", [(1 << 15, 1), (1 << 16, 0), (50_048, 1)])
def test_partition_of_ordered_inputs(ctx, order, S, layout):
    # 2^25 keys over 2^26 values in 1024 to 1341 buckets (the partition at
    # 1024 threads): ordered inputs bring whole tiles of one bucket, random
    # order a few keys of every bucket per tile
    n, M = 1 << 25, 1 << 26
    keys = gen.feistel(gen.SEED_BASE + 61, n, M)
    if order == "ascending":
        keys = np.sort(keys)
    elif order == "descending":
        keys = np.sort(keys)[::-1].copy()
    elif order == "runs":   # sorted runs of 5000 keys in random order of runs
        srt = np.sort(keys)
        cuts = np.arange(0, n, 5000)
        perm = gen.shuffle(62, np.arange(cuts.size, dtype=np.uint32))
        keys = np.concatenate([srt[cuts[i]: cuts[i] + 5000] for i in perm])
    check(ctx, keys, M - 1, path=bs.PATH_PARTITION, S=S, threads=512, layout=layout)


# wide partition tiles: 2^26 + k keys make 2049 or more 32 Ki-key tiles, so
# most CTAs take two or more (each next tile is copied in behind the current
# one) and the last tile is ragged; keys offset by one element are not
# 16-byte aligned and every tile is loaded by the threads instead
WIDE = dict(path=bs.PATH_PARTITION, threads=512, part_threads=1024, part_tile_keys=32768)
# the same tiles at 512 threads (16 Ki keys, two CTAs per SM)
WIDE512 = dict(path=bs.PATH_PARTITION, threads=512, part_threads=512, part_tile_keys=16384)


@pytest.mark.parametrize("S", [1 << 15, 50_048])
@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("offset", [0, 1])
def test_wide_partition_tiles(ctx, S, layout, offset):
    n, M = (1 << 26) + 12_345, 1 << 27
    keys = gen.feistel(gen.SEED_BASE + 71, n, M)
    check(ctx, keys, M - 1, S=S, layout=layout, offset=offset, **WIDE)


@pytest.mark.parametrize("S", [1 << 18, 300_032])
@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("offset", [0, 1])
def test_wide_partition_tiles_512(ctx, S, layout, offset):
    # 2^26 + k keys in 16 Ki-key tiles: 4097, so that most CTAs take two
    n, M = (1 << 26) + 4_321, 1 << 27
    keys = gen.feistel(gen.SEED_BASE + 73, n, M)
    check(ctx, keys, M - 1, S=S, layout=layout, offset=offset, **WIDE512)
    if layout == 1 and offset == 0:   # keys above max_value, and repeats
        check(ctx, keys, M - (1 << 20) - 1, S=S, layout=layout, **WIDE512)
        rep = keys.copy()
        rep[::997] = rep[3]
        check(ctx, rep, M - 1, S=S, layout=layout, **WIDE512)


@pytest.mark.parametrize("wide", [WIDE, WIDE512], ids=["1024", "512"])
def test_wide_partition_in_place(ctx, wide):
    # keys and output in one buffer: the plan takes the exact layout and the
    # context's own partition buffer, which the wide tiles fill
    n, M = (1 << 26) + 999, 1 << 27
    keys = gen.feistel(gen.SEED_BASE + 74, n, M)
    check(ctx, keys, M - 1, S=1 << 15, layout=1, inplace=True, **wide)


@pytest.mark.parametrize("layout", [0, 1])
def test_wide_partition_range_and_repeats(ctx, layout):
    n, M = (1 << 26) + 7, 1 << 27
    keys = gen.feistel(gen.SEED_BASE + 72, n, M)
    # keys above max_value are skipped and reported
    check(ctx, keys, M - (1 << 20) - 1, S=1 << 15, layout=layout, **WIDE)
    # repeated keys: the distinct prefix and DUPLICATE
    rep = keys.copy()
    rep[::1000] = rep[1]
    check(ctx, rep, M - 1, S=1 << 15, layout=layout, **WIDE)


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("persistent", [0, 1])
def test_repeats_spread_over_many_slices(ctx, layout, persistent):
    # repeated keys in many buckets: every slice after the first short one
    # is moved down to close the gaps; also in place
    keys = gen.uniform_with_replacement(31, 200_000, 1 << 20)
    for S in (4096, 1 << 16):
        check(ctx, keys, (1 << 20) - 1, path=bs.PATH_PARTITION, S=S, layout=layout, persistent=persistent)
        check(ctx, keys, (1 << 20) - 1, path=bs.PATH_PARTITION, S=S, layout=layout, persistent=persistent,
              inplace=True)
    # a single repeat near the end: only the last slices move
    keys = gen.floyd(32, 150_000, 1 << 20)
    keys[-1] = keys[0]
    check(ctx, keys, (1 << 20) - 1, path=bs.PATH_PARTITION, S=4096, layout=layout, persistent=persistent)


@pytest.mark.parametrize("name,strat", STRATS, ids=[x[0] for x in STRATS])
def test_key_range_skips_and_reports(ctx, name, strat):
    keys = gen.floyd(9, 20_000, 1 << 18)
    mv = (1 << 17) + 3   # about half the keys are out of range
    if strat["path"] == bs.PATH_FUSED:
        mv = (1 << 16) + 3
        keys = gen.floyd(9, 20_000, 1 << 17)
    check(ctx, keys, mv, **strat)


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
    for i in range(16):
        n, M = [(5000, 1 << 16), (70_000, 1 << 22), (3, 1 << 32), (200_000, 1 << 24)][i % 4]
        strat = [STRATS[1][1], STRATS[3][1], dict(), STRATS[2][1]][i % 4]
        check(ctx, gen.floyd(100 + i, n, M), M - 1, **strat)


def test_autotune_picks_a_correct_config(ctx, tmp_path):
    import torch
    keys_np = gen.floyd(13, 1 << 18, 1 << 22)
    keys = to_dev(keys_np)
    best = ctx.autotune(keys, (1 << 22) - 1, out=torch.empty_like(keys))
    assert best["path"] in ("fused", "partition", "global") and best["ms"] > 0
    got = ctx.get_config(1 << 18, (1 << 22) - 1)
    assert {k: got[k] for k in got if k != "ms"} == {k: best[k] for k in best if k != "ms"}
    check(ctx, keys_np, (1 << 22) - 1)
    p = str(tmp_path / "tune.json")
    ctx.tune_save(p)
    c2 = bs.Context(0)
    c2.tune_load(p)
    a2, a1 = c2.get_config(1 << 18, (1 << 22) - 1), ctx.get_config(1 << 18, (1 << 22) - 1)
    assert {k: a2[k] for k in a2 if k != "ms"} == {k: a1[k] for k in a1 if k != "ms"}
    c2.close()


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("summary", [0, 1])
def test_sparse_slices_summary_bitmap(ctx, layout, summary):
    # 16 slices of 2^20 values with ~190 keys each: sparse (summary bitmap)
    keys = gen.floyd(41, 3000, 1 << 24)
    check(ctx, keys, (1 << 24) - 1, path=bs.PATH_PARTITION, S=1 << 20, layout=layout, summary=summary)
    # a full 32-bit range with few keys
    keys = gen.feistel(42, 20_000, 1 << 32)
    check(ctx, keys, (1 << 32) - 1, path=bs.PATH_PARTITION, S=1 << 20, layout=layout, summary=summary)


@pytest.mark.parametrize("persistent", [0, 1])
def test_sparse_and_dense_slices_mixed(ctx, persistent):
    # dense lower half, a sprinkle of keys in the upper half: the CTAs meet
    # dense and sparse slices in turn (the cleared-bitmap bookkeeping)
    lo = gen.floyd(43, 400_000, 1 << 20)
    hi = (gen.floyd(44, 300, 1 << 23) + (1 << 23)).astype(np.uint32)
    keys = gen.shuffle(45, np.concatenate([lo, hi]))
    for S in (1 << 16, 1 << 18):
        check(ctx, keys, (1 << 24) - 1, path=bs.PATH_PARTITION, S=S, layout=1, persistent=persistent)
    check(ctx, keys, (1 << 24) - 1, path=bs.PATH_PARTITION, S=1 << 17, layout=0, threads=256)


def test_sparse_duplicates_and_in_place(ctx):
    keys = gen.uniform_with_replacement(46, 2000, 1 << 24)
    check(ctx, keys, (1 << 24) - 1, path=bs.PATH_PARTITION, S=1 << 20, layout=1)
    keys = gen.floyd(47, 2500, 1 << 22)
    check(ctx, keys, (1 << 22) - 1, path=bs.PATH_PARTITION, S=1 << 20, layout=1, inplace=True)
    check(ctx, gen.floyd(48, 5000, 1 << 20), (1 << 20) - 1, path=bs.PATH_FUSED)   # fused, sparse


@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffer_entry_point(ctx, pinned):
    """bitsort_host: keys in host memory, output and outcome back in host
    memory (page-locked or not), equal to the oracle; in place; duplicates."""
    import torch
    for n, M in ((100_000, 1 << 20), (300_001, 1 << 28), (0, 16)):
        keys_np = gen.keys(gen.SEED_BASE + 60 + n, n, M) if n else np.zeros(0, np.uint32)
        hk = torch.from_numpy(keys_np.view(np.int32).copy())
        ho = torch.empty(n, dtype=torch.int32)
        hr = torch.zeros(2, dtype=torch.int64)
        if pinned:
            hk, ho, hr = hk.pin_memory(), ho.pin_memory(), hr.pin_memory()
        s = torch.cuda.Stream()
        ctx.sort_host_async(hk, M - 1, ho, hr, stream=s)
        s.synchronize()
        want_st, want = oracle.bitmap_sort(keys_np, M - 1)
        assert int(hr[0]) == want_st and int(hr[1]) == want.size
        assert np.array_equal(ho.numpy().view(np.uint32)[:want.size], want)
    # in place in host memory, with a repeated key
    keys_np = gen.keys(gen.SEED_BASE + 61, 50_000, 1 << 24)
    keys_np[7] = keys_np[3]
    hk = torch.from_numpy(keys_np.view(np.int32).copy())
    hr = torch.zeros(2, dtype=torch.int64)
    ctx.sort_host_async(hk, (1 << 24) - 1, hk, hr)
    torch.cuda.synchronize()
    want_st, want = oracle.bitmap_sort(keys_np, (1 << 24) - 1)
    assert int(hr[0]) == want_st == bs.ERR_DUPLICATE and int(hr[1]) == want.size
    assert np.array_equal(hk.numpy().view(np.uint32)[:want.size], want)
