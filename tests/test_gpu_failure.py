"""Failure detection on the GPU without a fault: a bounded wait that can never
be satisfied must end with BITSORT_ERR_TIMEOUT, and the context must stay
usable afterwards."""
import numpy as np
import pytest

import gen
import paper_1312_0138_gb300 as bs
from gpu_util import gpu_sort, to_dev

pytestmark = pytest.mark.gpu


def test_stalled_predecessor_times_out_and_context_recovers():
    import time
    import torch
    ctx = bs.Context(0)
    ctx.set_wait_limit_ms(300)
    keys_np = gen.floyd(3, 50_000, 1 << 20)
    keys = to_dev(keys_np)
    out = torch.empty_like(keys)
    t0 = time.time()
    ctx.debug_stalled_launch(keys, (1 << 20) - 1, out)
    st, cnt = ctx.sync_status()
    took = time.time() - t0
    assert st == bs.ERR_TIMEOUT
    assert took < 30
    # the context reset its scratch: the next sorts are exact
    for path in (bs.PATH_PARTITION, bs.PATH_GLOBAL, bs.PATH_FUSED):
        st, cnt, got = gpu_sort(ctx, keys_np, (1 << 20) - 1, path=path)
        assert st == bs.OK and np.array_equal(got, np.sort(keys_np))
    ctx.close()
