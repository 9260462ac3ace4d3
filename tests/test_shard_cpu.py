"""Host logic of the sort spread over ranks by value range
(paper_1312_0138_gb300/shard.py) on CPU gloo ranks: the value ranges, the
two all-to-alls, the offsets.  The GPU operations are replaced by stand-ins
written here (grouping by owner and sorting with numpy), so only the
exchange and the bookkeeping are under test; tests/test_gpu_shard.py runs the
same function with the library's kernels."""
import os
import socket

import numpy as np
import pytest

import paper_1312_0138_gb300 as bs
from paper_1312_0138_gb300 import shard


class NumpyOps:
    """Stand-ins for the device operations, on CPU tensors."""

    def width(self, max_value, world):
        return bs.range_width(max_value, world)

    def split(self, keys, max_value, parts):
        import torch
        k = keys.numpy().view(np.uint32).astype(np.uint64)
        w = self.width(max_value, parts)
        keep = k <= max_value
        owner = np.minimum(k // w, parts - 1)
        order = np.argsort(owner[keep], kind="stable")
        grouped = k[keep][order].astype(np.uint32)
        counts = [int(c) for c in np.bincount(owner[keep].astype(np.int64), minlength=parts)]
        return torch.from_numpy(grouped.view(np.int32).copy()), counts

    def sort_span(self, keys, lo, hi):
        import torch
        k = keys.numpy().view(np.uint32)
        inr = (k >= lo) & (k <= hi)
        u = np.unique(k[inr])
        st = bs.OK if inr.all() and u.size == k.size else (bs.ERR_KEY_RANGE if not inr.all() else bs.ERR_DUPLICATE)
        return torch.from_numpy(u.view(np.int32).copy()), st, int(u.size)


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
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = keys_all[rank::world]
        res = shard.sort_range_sharded(torch.from_numpy(mine.view(np.int32).copy()), max_value, NumpyOps())
        np.save(os.path.join(outdir, f"r{rank}.npy"),
                np.array([res.count, res.offset, res.total, res.status, res.lo, res.hi], dtype=np.int64))
        np.save(os.path.join(outdir, f"k{rank}.npy"), res.out.numpy().view(np.uint32)[: res.count])
    finally:
        dist.destroy_process_group()


def run_ranks(world, keys_all, max_value, tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_rank, args=(world, _free_port(), keys_all, max_value, str(tmp_path)), nprocs=world, join=True)
    meta = [np.load(tmp_path / f"r{r}.npy") for r in range(world)]
    pieces = [np.load(tmp_path / f"k{r}.npy") for r in range(world)]
    return meta, pieces


def test_range_bounds_cover_the_values_once():
    for mv, g in [(99, 2), ((1 << 32) - 1, 2), ((1 << 32) - 1, 7), (1000, 3), (10, 16)]:
        b = shard.range_bounds(mv, g)
        w = bs.range_width(mv, g)
        assert w % 128 == 0 and w * g >= mv + 1
        covered = [v for lo, hi in b for v in ((lo, hi),) if hi >= lo]
        assert covered[0][0] == 0 and covered[-1][1] == mv
        for (lo0, hi0), (lo1, hi1) in zip(covered, covered[1:]):
            assert lo1 == hi0 + 1


@pytest.mark.parametrize("world", [2, 3])
def test_exchange_and_offsets_give_the_sorted_whole(tmp_path, world):
    import gen
    n, M = 50_000, 1 << 24
    keys = gen.feistel(77 + world, n, M)
    meta, pieces = run_ranks(world, keys, M - 1, tmp_path)
    whole = np.concatenate(pieces)
    assert np.array_equal(whole, np.sort(keys))
    off = 0
    for r, m in enumerate(meta):
        count, offset, total, status, lo, hi = (int(v) for v in m)
        assert status == bs.OK and offset == off and total == n
        assert pieces[r].size == count and (count == 0 or (pieces[r][0] >= lo and pieces[r][-1] <= hi))
        off += count


def test_repeats_across_ranks_reported_by_the_owner(tmp_path):
    import gen
    keys = gen.floyd(5, 20_000, 1 << 20)
    keys = np.concatenate([keys, keys[:1]])   # one key on two ranks
    meta, pieces = run_ranks(2, keys, (1 << 20) - 1, tmp_path)
    st = [int(m[3]) for m in meta]
    assert st.count(bs.ERR_DUPLICATE) == 1 and st.count(bs.OK) == 1
    assert np.array_equal(np.concatenate(pieces), np.unique(keys))
