"""Batched plans and the serving loop run again and again: every replay's
outcomes and outputs against the CPU oracle, for every batch policy the batch
autotuner may pick, on a non-blocking stream that starts work right after the
plan is built (a launch stream that does not wait for the legacy default
stream)."""
import numpy as np
import pytest

import gen
import oracle
import paper_1312_0138_gb300 as bs
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu

# the batch autotuner's sweep (bitsort_batch_autotune): path x slice x block x words per lane
POLICIES = [(p, s, t, w) for p in (bs.PATH_PARTITION, bs.PATH_GLOBAL) for s in (1 << 17, 1 << 18, 1 << 19, 1 << 20)
            for t in (256, 512) for w in (1, 2)]


@pytest.fixture(scope="module")
def ctx():
    c = bs.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def batch():
    """A mixed batch: uneven sizes and ranges (one fused slice up to many
    slices), plus the edge cases: empty, one key, duplicates, keys above
    max_value, the full 32-bit range; with the oracle's outcome of each."""
    spec = gen.batch_spec(77, 120, n_lo=1, n_hi=1 << 16, m_lo=1 << 8, m_hi=1 << 24)
    arrays = [(gen.floyd(770 + i, n, M), M - 1) for i, (n, M) in enumerate(spec)]
    arrays.append((np.zeros(0, np.uint32), 10))
    arrays.append((np.array([12345], np.uint32), 12345))
    arrays.append((gen.uniform_with_replacement(771, 40_000, 1 << 16), (1 << 16) - 1))
    arrays.append((gen.floyd(772, 30_000, 1 << 22), (1 << 21) + 3))
    arrays.append((gen.floyd(773, 1 << 14, 1 << 32), (1 << 32) - 1))
    arrays.append((gen.floyd(774, 1 << 18, 1 << 19), (1 << 19) - 1))   # density 1/2 across slices
    want = [oracle.bitmap_sort(k, mv) for k, mv in arrays]
    return arrays, want


def _run_and_check(plan, arrays, want, outs, stream, reps, label):
    for rep in range(reps):
        for o in outs:
            o.fill_(-1)
        plan.launch(stream=stream)
        res = plan.results(stream=stream)
        for i, ((k, mv), (st, cnt), (w_st, w)) in enumerate(zip(arrays, res, want)):
            assert (st, cnt) == (w_st, w.size), (label, rep, i, st, cnt, w_st, w.size)
            assert np.array_equal(to_host(outs[i])[:cnt], w), (label, rep, i)


@pytest.mark.parametrize("policy", POLICIES, ids=[f"p{p}-S{s >> 10}k-T{t}-w{w}" for p, s, t, w in POLICIES])
def test_every_autotuner_policy_replays_exactly(ctx, batch, policy):
    import torch
    arrays, want = batch
    path, S, T, wpl = policy
    ctx.set_batch_config(path, S, T, wpl, 0)
    try:
        keys = [to_dev(k) for k, _ in arrays]
        outs = [torch.empty_like(k) for k in keys]
        stream = torch.cuda.Stream()   # non-blocking: does not wait for the legacy default stream
        plan = ctx.plan([(k, mv, o) for k, (_, mv), o in zip(keys, arrays, outs)])
        _run_and_check(plan, arrays, want, outs, stream, 2, policy)
        plan.close()
        # one-shot batched call on the same stream, results on the device
        res = torch.zeros((len(arrays), 2), dtype=torch.int64, device="cuda")
        for o in outs:
            o.fill_(-1)
        ctx.batched([(k, mv, o) for k, (_, mv), o in zip(keys, arrays, outs)], results=res, stream=stream)
        stream.synchronize()
        r = res.cpu().numpy()
        for i, (w_st, w) in enumerate(want):
            assert (int(r[i, 0]) & 0xFFFFFFFF, int(r[i, 1])) == (w_st, w.size), (policy, i)
            assert np.array_equal(to_host(outs[i])[: w.size], w), (policy, i)
    finally:
        ctx.set_batch_config(bs.PATH_PARTITION, 1 << 19, 512, 1, 0)   # the default policy


def test_autotuned_policy_is_exact(ctx, batch):
    import torch
    arrays, want = batch
    keys = [to_dev(k) for k, _ in arrays]
    outs = [torch.empty_like(k) for k in keys]
    triples = [(k, mv, o) for k, (_, mv), o in zip(keys, arrays, outs)]
    try:
        ctx.batch_autotune(triples)
        plan = ctx.plan(triples)
        _run_and_check(plan, arrays, want, outs, torch.cuda.Stream(), 3, "autotuned")
        plan.close()
    finally:
        ctx.set_batch_config(bs.PATH_PARTITION, 1 << 19, 512, 1, 0)


def test_plain_sorts_on_fresh_nonblocking_streams():
    """A new context's first sort, and a global-bitmap sort that grows the
    bitmap, on a non-blocking stream right away: the zeroed scratch is in
    place before the kernels read it."""
    import torch
    for rep in range(4):
        c = bs.Context(0)
        s = torch.cuda.Stream()
        for n, M in [(100_000, 1 << 20), (1 << 20, 1 << 22), (1 << 18, 1 << 26)]:
            k = gen.floyd(900 + rep * 7 + n, n, M)
            kd = to_dev(k)
            out = c.sort_async(kd, M - 1, stream=s)
            st, cnt = c.sync_status(stream=s)
            assert st == bs.OK and cnt == n, (rep, n, M, st, cnt)
            assert np.array_equal(to_host(out), np.sort(k)), (rep, n, M)
        c.close()
