"""The sort spread over ranks by value range, with the library's kernels:
bitsort_range_split and bitsort_span against the CPU oracle, and two ranks
(processes sharing this one GPU, exchanging over gloo: no kernel of one rank
waits for the other's) whose pieces, in rank order, equal the oracle's sort
of all their keys element by element."""
import os
import socket

import numpy as np
import pytest

import gen
import oracle
import paper_1312_0138_gb300 as bs
from paper_1312_0138_gb300 import shard
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = bs.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("n,M,parts", [(100_000, 1 << 20, 2), (1_000_003, 1 << 32, 8), (5, 40, 3),
                                       (70_000, 1 << 24, 13), (1 << 20, 1 << 26, 1)])
def test_range_split_groups_by_owner(ctx, n, M, parts):
    import torch
    keys = gen.feistel(300 + parts, n, M)
    res = torch.zeros(2, dtype=torch.int64, device="cuda")
    out, counts = ctx.range_split_async(to_dev(keys), M - 1, parts, result=res)
    torch.cuda.synchronize()
    r = res.cpu().tolist()
    assert int(r[0]) & 0xFFFFFFFF == bs.OK and int(r[1]) == n
    w = bs.range_width(M - 1, parts)
    want = np.bincount(np.minimum(keys.astype(np.uint64) // w, parts - 1).astype(np.int64), minlength=parts)
    got_c = counts.cpu().numpy()
    assert np.array_equal(got_c, want)
    o = to_host(out)
    start = 0
    for g in range(parts):
        grp = o[start: start + got_c[g]]
        assert np.all(np.minimum(grp.astype(np.uint64) // w, parts - 1) == g), g
        start += got_c[g]
    assert np.array_equal(np.sort(o), np.sort(keys))   # every key once
    # the context's scratch is back at zero: a sort on it afterwards is exact
    st, cnt, srt = ctx.sort(to_dev(keys), M - 1)
    assert st == bs.OK and np.array_equal(to_host(srt), np.sort(keys))


def test_range_split_reports_keys_above_max_value(ctx):
    import torch
    keys = gen.floyd(31, 50_000, 1 << 20)
    mv = (1 << 19) - 1
    res = torch.zeros(2, dtype=torch.int64, device="cuda")
    out, counts = ctx.range_split_async(to_dev(keys), mv, 4, result=res)
    torch.cuda.synchronize()
    r = res.cpu().tolist()
    inr = keys[keys <= mv]
    assert int(r[0]) & 0xFFFFFFFF == bs.ERR_KEY_RANGE and int(r[1]) == inr.size
    assert int(counts.sum()) == inr.size
    assert np.array_equal(np.sort(to_host(out)[: inr.size]), np.sort(inr))


@pytest.mark.parametrize("lo,hi,n", [(1 << 30, (1 << 30) + (1 << 22) - 1, 1 << 20), (0, 999, 1000),
                                     ((1 << 32) - 5000, (1 << 32) - 1, 4000), (12345, 12345, 1)])
def test_span_sort_matches_oracle(ctx, lo, hi, n):
    import torch
    keys = (gen.floyd(7 + n, n, hi - lo + 1).astype(np.uint64) + lo).astype(np.uint32)
    res = torch.zeros(2, dtype=torch.int64, device="cuda")
    out = ctx.sort_span_async(to_dev(keys), lo, hi, result=res)
    torch.cuda.synchronize()
    r = res.cpu().tolist()
    want_st, want = oracle.bitmap_sort(keys, hi)   # keys >= lo: the plain sort up to hi gives the same array
    assert int(r[0]) & 0xFFFFFFFF == want_st == bs.OK and int(r[1]) == n
    assert np.array_equal(to_host(out), want)
    # a key below lo is outside the span
    bad = keys.copy()
    if lo > 0:
        bad[0] = lo - 1
        res.zero_()
        ctx.sort_span_async(to_dev(bad), lo, hi, result=res)
        torch.cuda.synchronize()
        assert int(res[0].item()) & 0xFFFFFFFF == bs.ERR_KEY_RANGE


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, keys_all, max_value, outdir):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c = bs.Context(0)
        mine = keys_all[rank::world]
        res = shard.sort_range_sharded(to_dev(mine), max_value, shard.DeviceOps(c))
        np.save(os.path.join(outdir, f"r{rank}.npy"),
                np.array([res.count, res.offset, res.total, res.status], dtype=np.int64))
        np.save(os.path.join(outdir, f"k{rank}.npy"), to_host(res.out)[: res.count])
        c.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("n,M", [(1 << 22, 1 << 26), (300_001, 1 << 32)])
def test_two_ranks_give_the_sorted_whole(tmp_path, n, M):
    import torch.multiprocessing as mp
    keys = gen.feistel(gen.SEED_BASE + 40, n, M)
    mp.spawn(_rank, args=(2, _free_port(), keys, M - 1, str(tmp_path)), nprocs=2, join=True)
    meta = [np.load(tmp_path / f"r{r}.npy") for r in range(2)]
    pieces = [np.load(tmp_path / f"k{r}.npy") for r in range(2)]
    want_st, want = oracle.bitmap_sort(keys, M - 1)
    assert want_st == bs.OK
    assert all(int(m[3]) == bs.OK for m in meta)
    assert int(meta[0][1]) == 0 and int(meta[1][1]) == int(meta[0][0]) and int(meta[1][2]) == n
    assert np.array_equal(np.concatenate(pieces), want)
