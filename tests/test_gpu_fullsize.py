"""Parity at the full sizes of the benchmarked workloads, in the launch
configuration the benchmark uses (the context's default / tuned plan)."""
import numpy as np
import pytest

import gen
import oracle
import paper_1312_0138_gb300 as bs
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = bs.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("n,M,method,cfg", [
    (1 << 24, 1 << 28, "floyd", 1),       # L2-resident bitmap, 64 MiB of keys
    (1 << 24, 1 << 32, "feistel", 2),     # sparse full 32-bit range
])
@pytest.mark.parametrize("strat", [None, (bs.PATH_PARTITION, 0), (bs.PATH_PARTITION, 1), (bs.PATH_GLOBAL, 0)],
                         ids=["default", "exact", "capacity", "global"])
def test_full_size_exact(ctx, n, M, method, cfg, strat):
    keys_np = gen.keys(gen.SEED_BASE + cfg, n, M, method)
    path = None if strat is None else strat[0]
    if path is not None:
        ctx.set_config(n, M - 1, path, layout=strat[1])
    st, cnt, out = ctx.sort(to_dev(keys_np), M - 1)
    if path is not None:
        ctx.set_config(n, M - 1, bs.PATH_AUTO)
    want_st, want = oracle.bitmap_sort(keys_np, M - 1)
    assert st == want_st == bs.OK and cnt == n
    assert np.array_equal(to_host(out), want)


def test_dense_full_range_2e31_properties(ctx):
    """n = 2^31 distinct keys from [0, 2^32) (density 1/2): the keys are
    pi(0..n-1) for a seeded bijection pi, so the output is the sorted image
    iff it has length n, is strictly increasing and every value v has
    pi^-1(v) < n.  All three are checked on every element."""
    import torch
    n, M = 1 << 31, 1 << 32
    keys_np = gen.feistel(gen.SEED_BASE + 2, n, M)
    keys = to_dev(keys_np)
    st, cnt, out = ctx.sort(keys, M - 1, out=torch.empty_like(keys))
    assert st == bs.OK and cnt == n
    del keys
    chunk = 1 << 28
    for s in range(0, n, chunk):
        c = out[s: s + chunk + 1].to(torch.int64) & 0xFFFFFFFF
        assert bool((c[1:] > c[:-1]).all()), s
    host = to_host(out)
    del out
    inv = gen.feistel_inverse(gen.SEED_BASE + 2, M, host)
    assert int(inv.max()) < n


@pytest.mark.parametrize("n,M,kind", [
    (1 << 24, 1 << 28, "distinct"),    # the benchmark's keys
    (1 << 24, 1 << 20, "repeat"),      # 16 keys per value on average
    (1 << 24, 1 << 32, "repeat"),      # full 32-bit values, four passes of 8 bits
])
def test_multiset_full_size(ctx, n, M, kind):
    """The multiset path (Algorithm 1's stable bit splits) at the benchmark's
    size, compared with the CPU oracle's Algorithm 1 element by element."""
    if kind == "distinct":
        keys_np = gen.keys(gen.SEED_BASE + 1, n, M, "floyd")
    else:
        keys_np = gen.uniform_with_replacement(gen.SEED_BASE + 90, n, M)
    st, cnt, out = ctx.multiset(to_dev(keys_np), M - 1)
    assert st == bs.OK and cnt == n
    assert np.array_equal(to_host(out), oracle.paper_sort_u32(keys_np))
