"""One sort spread over several GPUs by value range (host orchestration).

The paper's problem is one array and one ascending result (Section V,
BitwiseSort).  With G ranks, each holding a share of the keys, rank g owns
the values [g*W, (g+1)*W), W = bitsort_range_width(max_value, G):

1. every rank groups its keys by owner on its GPU (C entry point
   bitsort_range_split);
2. the ranks exchange the G group sizes and then the groups (two
   all-to-alls through torch.distributed: NCCL moves device tensors, gloo
   host copies);
3. every rank sorts the keys it received, which lie in its own range, on
   its GPU (C entry point bitsort_span);
4. an all-gather of the G output sizes gives every rank the offset of its
   piece in the sorted array.

Rank g's output is then the g-th piece of the sorted whole.  The sorting and
the grouping run in the library's kernels; this module only moves tensors
between ranks and computes offsets.  The device operations are passed in as
an object (`ops`), so that the exchange logic can also run on CPU ranks
with stand-in operations in tests.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional


def range_bounds(max_value: int, world: int, width: Optional[int] = None):
    """[(lo, hi)] inclusive value range of each rank (hi < lo: an empty range,
    where the ranks outnumber the values)."""
    M = max_value + 1
    if width is None:
        from . import range_width
        width = range_width(max_value, world)
    out = []
    for g in range(world):
        lo = g * width
        hi = min((g + 1) * width, M) - 1
        out.append((lo, hi))
    return out


@dataclass
class ShardResult:
    out: object          # this rank's piece of the sorted array (device tensor, `count` keys)
    count: int           # keys in this rank's piece
    offset: int          # index of the piece's first key in the sorted whole
    total: int           # keys in the sorted whole
    status: int          # the local sort's status (OK, KEY_RANGE, DUPLICATE)
    lo: int              # the rank's value range
    hi: int


class DeviceOps:
    """The library's kernels on one context (the default `ops`)."""

    def __init__(self, ctx, stream=None):
        self.ctx = ctx
        self.stream = stream

    def width(self, max_value: int, world: int) -> int:
        from . import range_width
        return range_width(max_value, world)

    def split(self, keys, max_value: int, parts: int):
        """(grouped keys, list of `parts` group sizes)."""
        grouped, counts = self.ctx.range_split_async(keys, max_value, parts, stream=self.stream)
        return grouped, [int(c) for c in counts.cpu().tolist()]

    def sort_span(self, keys, lo: int, hi: int):
        """(sorted keys, status, count) of keys in [lo, hi]."""
        import torch
        from . import OK
        if keys.numel() == 0:
            return keys, OK, 0
        res = torch.zeros(2, dtype=torch.int64, device=keys.device)
        out = self.ctx.sort_span_async(keys, lo, hi, result=res, stream=self.stream)
        r = res.cpu().tolist()
        return out, int(r[0]) & 0xFFFFFFFF, int(r[1])


def sort_range_sharded(keys, max_value: int, ops, group=None) -> ShardResult:
    """Collective over `group` (every rank calls it): the ranks' keys together
    form one array of distinct values in [0, max_value]; returns this rank's
    piece of its sorted form.  `keys` is a tensor of int32 / uint32 (bit
    patterns of uint32 keys) on the device `ops` works on."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    width = ops.width(max_value, world)
    bounds = range_bounds(max_value, world, width)
    lo, hi = bounds[rank]

    # 1. group by owner
    grouped, send_counts = ops.split(keys, max_value, world)

    # 2. exchange sizes, then keys; gloo moves host tensors
    host = dist.get_backend(group) == "gloo"
    dev = keys.device
    cdev = torch.device("cpu") if host else dev
    send_c = torch.tensor(send_counts, dtype=torch.int64, device=cdev)
    recv_c = torch.empty(world, dtype=torch.int64, device=cdev)
    dist.all_to_all_single(recv_c, send_c, group=group)
    recv_counts: List[int] = [int(c) for c in recv_c.tolist()]
    send_t = grouped[: sum(send_counts)]
    send_t = send_t.cpu() if host else send_t
    recv_t = torch.empty(sum(recv_counts), dtype=keys.dtype, device=cdev)
    dist.all_to_all_single(recv_t, send_t, recv_counts, send_counts, group=group)
    mine = recv_t.to(dev) if host else recv_t

    # 3. sort this rank's range
    if hi < lo:   # an empty range (more ranks than values): nothing can arrive
        from . import OK
        out, status, count = mine, OK, 0
    else:
        out, status, count = ops.sort_span(mine, lo, hi)

    # 4. offsets of the pieces
    cnt = torch.tensor([count], dtype=torch.int64, device=cdev)
    all_c = [torch.empty(1, dtype=torch.int64, device=cdev) for _ in range(world)]
    dist.all_gather(all_c, cnt, group=group)
    sizes = [int(c.item()) for c in all_c]
    return ShardResult(out=out, count=count, offset=sum(sizes[:rank]), total=sum(sizes), status=status,
                       lo=lo, hi=hi)
