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


def _check_feistel_output(out_dev, seed, n, M):
    """Length n, strictly increasing (on the device), and every value v has
    pi^-1(v) < n for the seeded bijection pi that made the keys: together, the
    output is the sorted key set."""
    import torch
    c = out_dev[:n].to(torch.int64) & 0xFFFFFFFF
    assert n < 2 or bool((c[1:] > c[:-1]).all())
    host = to_host(out_dev)[:n]
    assert n == 0 or int(gen.feistel_inverse(seed, M, host).max()) < n


def test_batched_full_size(ctx):
    """The benchmark's batch (4096 arrays, 2.07 G keys, seeds and sizes as
    timed) in one persistent launch with the default batch policy, replayed
    three times from its CUDA graph (the first replay on a non-blocking
    stream that starts right after the plan is built): every outcome, every
    output by its three properties, and a sample of arrays element by
    element against the oracle, after every replay."""
    import torch
    seed0 = gen.SEED_BASE
    spec = gen.batch_spec(seed0 + 3, 4096)
    keys_np = [gen.feistel(seed0 + 7 * i, n, M) for i, (n, M) in enumerate(spec)]
    keys = [to_dev(k) for k in keys_np]
    outs = [torch.empty_like(k) for k in keys]
    plan = ctx.plan([(k, M - 1, o) for k, (n, M), o in zip(keys, spec, outs)])
    side = torch.cuda.Stream()
    wants = {i: oracle.bitmap_sort(keys_np[i], spec[i][1] - 1) for i in range(0, 4096, 97)}
    for rep in range(3):
        for o in outs:
            o.fill_(-1)
        torch.cuda.synchronize()
        stream = side if rep == 0 else None
        plan.launch(stream=stream)
        res = plan.results(stream=stream)
        for i, ((n, M), (st, cnt)) in enumerate(zip(spec, res)):
            assert st == bs.OK and cnt == n, (rep, i, st, cnt, n)
            _check_feistel_output(outs[i], seed0 + 7 * i, n, M)
        for i, (want_st, want) in wants.items():
            assert want_st == bs.OK and np.array_equal(to_host(outs[i]), want), (rep, i)
    plan.close()


def test_served_full_size(ctx):
    """The benchmark's saturated serving run (300 Poisson requests, n up to
    2^26, max_value up to 2^32 - 1, 40 GiB budget, 4 streams), submitted
    twice to one server: every request's outcome and output in both rounds,
    and a sample element by element against the oracle."""
    import torch
    seed0 = gen.SEED_BASE
    spec = gen.serve_spec(seed0 + 4, 300, rate_hz=1e6)
    reqs = []
    for i, (_, n, M) in enumerate(spec):
        k = gen.feistel(seed0 + 11 * i, n, M)
        reqs.append((k, M - 1, to_dev(k)))
    wants = {i: oracle.bitmap_sort(reqs[i][0], reqs[i][1]) for i in range(0, 300, 37)}
    srv = bs.Server(0, budget_bytes=40 << 30, max_inflight=4)
    outs = [torch.empty_like(kd) for _, _, kd in reqs]
    for rnd in range(2):
        for o in outs:
            o.fill_(-1)
        torch.cuda.synchronize()
        tickets = [srv.submit(kd, mv, o) for (_, mv, kd), o in zip(reqs, outs)]
        for i, t in enumerate(tickets):
            st, cnt, _ = srv.wait(t)
            n, M = spec[i][1], spec[i][2]
            assert st == bs.OK and cnt == n, (rnd, i, st, cnt, n, M)
        for i in range(300):
            _check_feistel_output(outs[i], seed0 + 11 * i, spec[i][1], spec[i][2])
        for i, (want_st, want) in wants.items():
            assert want_st == bs.OK and np.array_equal(to_host(outs[i]), want), (rnd, i)
    srv.close()
