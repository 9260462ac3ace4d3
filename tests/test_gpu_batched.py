"""Batched sorts (one persistent launch, CUDA-graph replay) and the serving
loop: every array's output equals the oracle's, and equals the output of the
same array sorted alone."""
import numpy as np
import pytest

import gen
import oracle
import paper_1312_0138_gb300 as bs
from gpu_util import gpu_sort, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = bs.Context(0)
    yield c
    c.close()


def make_batch(seed, count, n_hi=1 << 16, m_hi=1 << 22):
    spec = gen.batch_spec(seed, count, n_lo=1, n_hi=n_hi, m_lo=1 << 6, m_hi=m_hi)
    arrays = []
    for i, (n, M) in enumerate(spec):
        arrays.append((gen.floyd(seed * 7919 + i, n, M), M - 1))
    return arrays


def test_batched_matches_oracle_and_replays(ctx):
    import torch
    arrays = make_batch(1, 300)
    arrays.append((np.zeros(0, np.uint32), 100))                     # empty array
    arrays.append((gen.floyd(5, 1 << 18, 1 << 32), (1 << 32) - 1))   # sparse full range
    arrays.append((gen.uniform_with_replacement(6, 3000, 4096), 4095))  # duplicates
    keys = [to_dev(k) for k, _ in arrays]
    outs = [torch.full_like(k, -1) for k in keys]
    plan = ctx.plan([(k, mv, o) for k, (_, mv), o in zip(keys, arrays, outs)])
    for rep in range(3):
        for o in outs:
            o.fill_(-1)
        plan.launch()
        res = plan.results()
        for i, ((k, mv), o, (st, cnt)) in enumerate(zip(arrays, outs, res)):
            want_st, want = oracle.bitmap_sort(k, mv)
            assert st == want_st and cnt == want.size, (rep, i, st, want_st)
            assert np.array_equal(to_host(o)[:cnt], want), (rep, i)
    plan.close()


def test_batched_in_place_and_one_shot(ctx):
    import torch
    arrays = make_batch(2, 64, n_hi=1 << 14)
    keys = [to_dev(k) for k, _ in arrays]
    res = torch.zeros((len(arrays), 2), dtype=torch.int64, device="cuda")
    ctx.batched([(k, mv, k) for k, (_, mv) in zip(keys, arrays)], results=res)   # out == keys
    torch.cuda.synchronize()
    r = res.cpu().numpy()
    for i, (k, mv) in enumerate(arrays):
        want_st, want = oracle.bitmap_sort(k, mv)
        assert int(r[i, 0]) & 0xFFFFFFFF == want_st and int(r[i, 1]) == want.size
        assert np.array_equal(to_host(keys[i])[: want.size], want)


def test_batch_equals_alone(ctx):
    import torch
    arrays = make_batch(3, 40, n_hi=1 << 17, m_hi=1 << 24)
    keys = [to_dev(k) for k, _ in arrays]
    outs = [torch.empty_like(k) for k in keys]
    plan = ctx.plan([(k, mv, o) for k, (_, mv), o in zip(keys, arrays, outs)])
    plan.launch()
    res = plan.results()
    for i, (k, mv) in enumerate(arrays):
        st, cnt, alone = gpu_sort(ctx, k, mv)
        assert (st, cnt) == res[i]
        assert np.array_equal(to_host(outs[i])[:cnt], alone)
    plan.close()


def test_server_results_alone_and_in_the_mix(ctx):
    import torch
    srv = bs.Server(0, budget_bytes=1 << 30, max_inflight=3)
    spec = gen.serve_spec(4, 120, rate_hz=1e9, n_lo=1 << 4, n_hi=1 << 18, m_lo=1 << 10, m_hi=1 << 32)
    reqs = []
    for i, (_, n, M) in enumerate(spec):
        k = gen.keys(1000 + i, n, M)
        kd = to_dev(k)
        reqs.append((k, M - 1, kd, torch.empty_like(kd)))
    tickets = [srv.submit(kd, mv, od) for (_, mv, kd, od) in reqs]
    lat = []
    for t, (k, mv, kd, od) in zip(tickets, reqs):
        st, cnt, l = srv.wait(t)
        lat.append(l)
        want_st, want = oracle.bitmap_sort(k, mv)
        assert st == want_st and cnt == want.size
        mixed = to_host(od)[:cnt]
        assert np.array_equal(mixed, want)
        st2, cnt2, alone = gpu_sort(ctx, k, mv)
        assert (st2, cnt2) == (st, cnt) and np.array_equal(alone, mixed)
    stats = srv.stats()
    assert stats["completed"] == len(reqs)
    assert stats["batches"] >= 1
    assert all(x > 0 for x in lat)
    srv.close()


def test_server_budget_admission(ctx):
    import torch
    srv = bs.Server(0, budget_bytes=1 << 20, max_inflight=2)
    big = to_dev(gen.floyd(1, 10, 1 << 30))
    with pytest.raises(bs.BitsortError) as e:
        srv.submit(big, (1 << 30) - 1, torch.empty_like(big))   # bitmap alone is 128 MiB
    assert e.value.status == bs.ERR_BUDGET
    # many requests that only fit a few at a time all complete
    ks = [gen.floyd(50 + i, 20_000, 1 << 20) for i in range(20)]   # 208 KiB each
    dev = [(to_dev(k), None) for k in ks]
    tickets = []
    for kd, _ in dev:
        od = torch.empty_like(kd)
        tickets.append((srv.submit(kd, (1 << 20) - 1, od), od))
    for (t, od), k in zip(tickets, ks):
        st, cnt, _ = srv.wait(t)
        assert st == bs.OK and np.array_equal(to_host(od), np.sort(k))
    srv.close()


def test_server_budget_counts_plain_scratch():
    # 2^20 keys over 2^28 values: its plain sort asks its stream's context for
    # a capacity partition buffer of about 1.07 GB (304 buckets of 883,072
    # entries), held afterwards; with that, it fits a 2 GiB budget but not a
    # 1 GiB one (its bitmap and output alone are 36 MiB)
    import torch
    keys_np = gen.floyd(77, 1 << 20, 1 << 28)
    kd = to_dev(keys_np)
    small = bs.Server(0, budget_bytes=1 << 30, max_inflight=2)
    with pytest.raises(bs.BitsortError) as e:
        small.submit(kd, (1 << 28) - 1, torch.empty_like(kd))
    assert e.value.status == bs.ERR_BUDGET
    small.close()
    srv = bs.Server(0, budget_bytes=2 << 30, max_inflight=2)
    outs = [torch.empty_like(kd) for _ in range(3)]
    tickets = [srv.submit(kd, (1 << 28) - 1, o) for o in outs]
    want = np.sort(keys_np)
    for t, o in zip(tickets, outs):
        st, cnt, _ = srv.wait(t)
        assert st == bs.OK and cnt == keys_np.size
        assert np.array_equal(to_host(o), want)
    srv.close()
