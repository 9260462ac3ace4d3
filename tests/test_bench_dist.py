"""The benchmark's multi-process path on CPU: two ranks over gloo (no GPU).
Each rank sorts its own array (its own seed), the ranks meet at a barrier,
the job time is the slowest rank's and the job throughput counts every
rank's keys; the reference arm runs on rank 0 alone."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, ws, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      CUDA_VISIBLE_DEVICES="")   # CPU ranks (gloo) even on a machine with a GPU
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    got_ws, got_rank, _ = bench.dist_init()
    assert (got_ws, got_rank) == (ws, rank)
    assert dist.get_backend() == "gloo"
    bench.barrier(ws)
    slowest = bench.max_over_ranks(ws, 1.0 + rank)          # rank r "took" 1 + r ms
    w = dict(cfg=0, n=5000, M=1 << 16, method="floyd")
    keys = bench.make_keys(w, rank)
    q.put((rank, slowest, keys.astype(np.int64).tolist()))
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_ranks_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        rank, slowest, keys = q.get(timeout=240)
        out[rank] = (slowest, keys)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    # the job time is the slowest rank's on every rank
    assert out[0][0] == out[1][0] == 2.0
    # each rank sorts its own distinct, in-range keys (its own seed)
    k0, k1 = np.array(out[0][1]), np.array(out[1][1])
    for k in (k0, k1):
        assert k.size == 5000 and np.unique(k).size == 5000 and k.min() >= 0 and k.max() < (1 << 16)
    assert not np.array_equal(k0, k1)


def test_job_throughput_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench
    # 2 ranks x 2^24 keys in 0.5 ms (slowest rank) = 67.1 Gkeys/s
    assert bench.job_gkeys_s(2, 1 << 24, 0.5) == pytest.approx(2 * (1 << 24) / 0.5e-3 / 1e9)
    assert bench.job_gkeys_s(1, 1000, 1.0) == pytest.approx(1e-3)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench
    w = dict(cfg=0, n=1000, M=1 << 16, method="floyd", desc="tiny")

    class Args:
        steps, warmup, cpu_budget = 1, 0, 1.0

    bench.run_reference(Args, w, 2, 1)      # rank 1 of 2: no work, no line
    assert capsys.readouterr().out == ""
