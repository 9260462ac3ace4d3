"""Helpers shared by the GPU tests: device tensors of uint32 keys and the
library call through the C ABI."""
import numpy as np

import paper_1312_0138_gb300 as bs


def to_dev(a: np.ndarray):
    import torch
    a = np.ascontiguousarray(a, dtype=np.uint32)
    return torch.from_numpy(a.view(np.int32)).cuda()


def to_host(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def gpu_sort(ctx, keys_np, max_value, path=None, S=0, threads=0, inplace=False, offset=0, **cfg):
    """Sort on the GPU through bitsort_ex; returns (status, count, out[:count]).
    With `path`, the size class is first set to that configuration (extra
    keyword arguments: words_per_lane, stage, layout, persistent)."""
    import torch
    n = keys_np.size
    if path is not None:
        ctx.set_config(max(n, 1), max_value, path, S, threads, **cfg)
    if offset:
        # keys and out start `offset` elements into their allocations (unaligned)
        kbuf = to_dev(np.concatenate([np.zeros(offset, np.uint32), keys_np]))
        keys = kbuf[offset:]
        obuf = torch.empty(n + offset, dtype=torch.int32, device="cuda")
        out = obuf[offset:]
    else:
        keys = to_dev(keys_np)
        out = keys if inplace else torch.empty_like(keys)
    st, cnt, out = ctx.sort(keys, max_value, out=out)
    if path is not None:
        ctx.set_config(max(n, 1), max_value, bs.PATH_AUTO)
    if st == bs.ERR_TIMEOUT:
        raise AssertionError("device wait timed out")
    return st, cnt, to_host(out)[:cnt]
