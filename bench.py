"""Benchmark of the GB300 bitmap sort.

Default workload: the largest single-array configuration, one array of
n = 2^31 distinct uint32 keys over the full 32-bit range [0, 2^32) (density
1/2; 8 GiB of keys in, 8 GiB out, a 512 MiB bitmap), the keys pi(0..n-1) of a
seeded Feistel bijection pi (a stand-in for sampling without replacement).
One step = one sort of the whole array (every step of the path: range check,
partition, scatter, popcount, offsets, emission) through the C ABI call
`bitsort_ex`, inputs already resident in HBM.  L2 is flushed between timed
steps (a 512 MiB write and a 512 MiB read, outside the timed events); the
arrays are also far larger than L2.

Other workloads (--workload): c0 (n=1e5, M=2^20), c1 (n=2^24, M=2^28),
c2b (n=2^24, M=2^32), batched (4096 arrays, one launch, graph replay),
served (Poisson arrivals through the serving loop).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank sorts its own array (weak scaling, no collective on
the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sorted Gkeys/s and % HBM roofline, plain vs batched/served; p50/p99 latency"
SEED = 0x13120138

WORKLOADS = {
    "c0": dict(n=100_000, M=1 << 20, method="floyd", cfg=0,
               desc="plain bitsort, one array: n=100000 distinct uint32 from [0,2^20), max_value=2^20-1"),
    "c1": dict(n=1 << 24, M=1 << 28, method="floyd", cfg=1,
               desc="plain bitsort, one array: n=2^24 distinct uint32 from [0,2^28) (density 1/16), "
                    "max_value=2^28-1, bitmap 32 MiB"),
    "c2a": dict(n=1 << 31, M=1 << 32, method="feistel", cfg=2,
                desc="plain bitsort, dense full range: n=2^31 distinct uint32 from [0,2^32) (Feistel "
                     "permutation stand-in for sampling without replacement)"),
    "c2b": dict(n=1 << 24, M=1 << 32, method="feistel", cfg=2,
                desc="plain bitsort, sparse full range: n=2^24 distinct uint32 from [0,2^32) (density 1/256)"),
}


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def engine_source_hash():
    """Hash of the kernel sources (the device code the counters describe),
    comments and blank space left out so that only code changes count."""
    import re
    h = hashlib.sha256()
    for f in ("engine.cu", "engine.h", "ptx.cuh"):
        with open(os.path.join(ROOT, "paper_1312_0138_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(f.encode() + " ".join(text.split()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(workload):
    """DRAM bytes per launch from the committed ncu summary, only if it was
    taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        e = d.get(workload)
        if e and e.get("source_hash") == engine_source_hash():
            return e.get("dram_bytes_per_launch")
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, value):
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gkeys_s(ws, n_per_rank, ms_max):
    """Whole-job throughput: the keys all ranks sorted (each rank its own
    array of n_per_rank keys, weak scaling) over the slowest rank's time."""
    return ws * n_per_rank / (ms_max * 1e-3) / 1e9


def make_keys(w, rank):
    import gen
    return gen.keys(SEED + w["cfg"] + 1000 * rank, w["n"], w["M"], w["method"])


# ------------------------------------------------------------ CPU oracle
def time_oracle(keys_np, max_value, budget_s=10.0, max_keys=None):
    """Oracle on the host (single thread) on a bounded sample: whole runs of
    the array (or of its first max_keys keys) until budget_s has elapsed."""
    import oracle
    sample = keys_np if max_keys is None or keys_np.size <= max_keys else keys_np[:max_keys]
    runs, t_total = 0, 0.0
    while t_total < budget_s or runs == 0:
        t0 = time.perf_counter()
        st, out = oracle.bitmap_sort(sample, max_value)
        t_total += time.perf_counter() - t0
        runs += 1
        if runs >= 50:
            break
    return {"value": runs * sample.size / t_total / 1e9, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
            "sample": f"{runs} single-threaded oracle run(s) over {sample.size} keys of the workload "
                      f"(max_value={max_value}), {t_total:.1f} s"}


def sample_keys(w, rank, max_keys):
    """The workload's first max_keys keys (all of them when it has fewer).
    Feistel keys are pi(0), pi(1), ...: the first k keys of the array are the
    k keys the generator gives for n = k."""
    import gen
    if max_keys is None or w["n"] <= max_keys:
        return make_keys(w, rank)
    if w["method"] == "feistel":
        return gen.keys(SEED + w["cfg"] + 1000 * rank, max_keys, w["M"], "feistel")
    return make_keys(w, rank)[:max_keys]


def run_reference(args, w, ws, rank):
    if rank != 0:
        return
    max_keys = 1 << 24 if w["n"] > (1 << 24) else None
    keys_np = sample_keys(w, rank, max_keys)
    M = w["M"]
    per_step = []
    for _ in range(args.warmup + args.steps):
        r = time_oracle(keys_np, M - 1, budget_s=0.0, max_keys=max_keys)
        per_step.append(r)
    vals = [r["value"] for r in per_step[args.warmup:]]
    v = float(np.median(vals))
    n_step = min(w["n"], max_keys or w["n"])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Gkeys/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": n_step / (v * 1e9) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": w["desc"], "n": w["n"], "max_value": M - 1},
            "cpu_baseline": {"value": v, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
                             "sample": f"each step one single-threaded oracle run over {n_step} keys"},
            "e2e": {"value": v, "unit": "Gkeys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- GPU arm
def run_plain(args, w, ws, rank, local):
    import torch
    import paper_1312_0138_gb300 as bs

    dev = local if torch.cuda.is_available() else 0
    torch.cuda.set_device(dev)
    torch.cuda.set_stream(torch.cuda.Stream())   # a non-default stream: phases chain by programmatic launch
    bs.load()
    ctx = bs.Context(dev)
    keys_np = make_keys(w, rank)
    n, M = w["n"], w["M"]
    keys = torch.from_numpy(keys_np.view(np.int32)).cuda()
    out = torch.empty_like(keys)
    if args.tune:
        ctx.autotune(keys, M - 1, out=out)
    if args.path:
        ctx.set_config(n, M - 1, {"fused": 1, "partition": 2, "global": 3}[args.path], args.slice, args.threads,
                       words_per_lane=args.wpl, stage=args.stage, layout=args.layout, persistent=args.persistent,
                       emit=args.emit, part_stream=args.part_stream, part_threads=args.part_threads,
                       part_tile_keys=args.part_tile_keys)
    cfg = ctx.get_config(n, M - 1)
    flush = L2Flush(args.flush)
    stream = torch.cuda.current_stream()

    # correctness of the measured configuration (one sort, checked on device)
    st, cnt, _ = ctx.sort(keys, M - 1, out=out)
    assert st == bs.OK and cnt == n, (st, cnt)

    for _ in range(args.warmup):
        flush.fill_(1)
        ctx.sort_async(keys, M - 1, out=out)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches0 = ctx.kernel_launches()
    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)                      # evict keys/out/bitmap from L2
        starts[i].record(stream)
        ctx.sort_async(keys, M - 1, out=out)
        ends[i].record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    launches = ctx.kernel_launches() - launches0
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms_step = float(np.mean(ms))
    ms_step_max = max_over_ranks(ws, ms_step)
    st, cnt = ctx.sync_status()
    assert st == bs.OK and cnt == n

    value = job_gkeys_s(ws, n, ms_step_max)
    peak, peak_kind = read_peaks()
    algo_bytes = 8 * n + M // 4
    path_achieved = algo_bytes / (ms_step * 1e-3) / 1e9

    # per-kernel event times (second pass, same flushes): the dominant kernel
    phase_steps = min(args.steps, 200)
    ctx.set_phase_timing(True)
    per_kind = {}
    for i in range(phase_steps):
        flush.fill_(i & 0xFF)
        ctx.sort_async(keys, M - 1, out=out)
        for kind, t in ctx.phase_times():
            per_kind.setdefault(kind, []).append(t)
    ctx.set_phase_timing(False)
    kind_ms = {k: float(np.mean(v)) for k, v in per_kind.items()}
    dom = max(kind_ms, key=kind_ms.get)
    # algorithmic bytes of one launch of each kernel: 8 B per key (read + write
    # of a 4-byte key) and, for the kernels that build and read the bitmap,
    # M/8 + M/8 bitmap bytes
    kernel_bytes = {"hist": 4 * n, "part": 8 * n, "parts": 8 * n, "partw": 8 * n, "gscatter": 4 * n + M // 8,
                    "gscan": 4 * n + M // 8, "bucket": 8 * n + M // 4, "persistent": 8 * n + M // 4}
    # the bytes each kernel must move through L2 / HBM: the bucket kernel
    # builds and reads its bitmap slices in shared memory (M/4 never leaves
    # the SM; sparse slices skip most of it through the summary bitmap), the
    # global-bitmap kernels really move their bitmap bytes through L2
    kernel_hbm_bytes = {"hist": 4 * n, "part": 8 * n, "parts": 8 * n, "partw": 8 * n, "gscatter": 4 * n + M // 8,
                        "gscan": 4 * n + M // 8, "bucket": 8 * n, "persistent": 8 * n}
    dom_bytes = kernel_bytes.get(dom, algo_bytes)
    dom_hbm_bytes = kernel_hbm_bytes.get(dom, 8 * n)
    achieved = dom_bytes / (kind_ms[dom] * 1e-3) / 1e9
    hbm_achieved = dom_hbm_bytes / (kind_ms[dom] * 1e-3) / 1e9

    # end to end through the host-buffer entry point (bitsort_host): every
    # step copies its keys from pinned host memory, sorts, and copies the
    # output and the outcome back.  Consecutive steps rotate over three
    # streams, each with its own context: a stream runs its step's copy in,
    # sort and copy out one after the other, so with three of them in flight
    # the copies of one step overlap the sort and the copies of the others
    # (the copy engines work in both directions at once).
    e2e_steps = max(3, min(args.steps, args.e2e_steps))
    hkeys = torch.from_numpy(keys_np.view(np.int32)).pin_memory()
    nl = 3
    lanes = []
    for li in range(nl):
        lanes.append(dict(ctx=ctx if li == 0 else bs.Context(local), stream=stream if li == 0 else torch.cuda.Stream(),
                          hout=torch.empty(n, dtype=torch.int32).pin_memory(),
                          hres=torch.zeros(2, dtype=torch.int64).pin_memory()))
    for i in range(2 * nl):
        ln = lanes[i % nl]
        ln["ctx"].sort_host_async(hkeys, M - 1, ln["hout"], ln["hres"], stream=ln["stream"])
    torch.cuda.synchronize()
    barrier(ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for ln in lanes[1:]:
        ln["stream"].wait_event(e0)
    for i in range(e2e_steps):
        ln = lanes[i % nl]
        ln["ctx"].sort_host_async(hkeys, M - 1, ln["hout"], ln["hres"], stream=ln["stream"])
    for ln in lanes[1:]:
        done = torch.cuda.Event()
        done.record(ln["stream"])
        stream.wait_event(done)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(ws, e0.elapsed_time(e1) / e2e_steps)
    for ln in lanes:
        assert int(ln["hres"][0]) & 0xFFFFFFFF == bs.OK and int(ln["hres"][1]) == n
        assert bool(np.all(np.diff(ln["hout"].numpy().view(np.uint32)[:1 << 20].astype(np.int64)) > 0))
    for ln in lanes[1:]:
        ln["ctx"].close()
    link = time_host_link(hkeys, lanes[0]["hout"], out, stream)
    link["e2e_gbs"] = (8 * n + 16) / (e2e_ms * 1e-3) / 1e9   # bytes each rank moves per step / step time

    comparison = None
    if not args.no_cub:
        comparison = {"cub": time_cub(keys, M, flush, stream, args.steps),
                      "multiset": time_multiset(ctx, keys, M, flush, stream, args.steps, 0, peak),
                      "multiset_1bit": time_multiset(ctx, keys, M, flush, stream, 3, 1, peak)}

    if rank != 0:
        return
    cpu = time_oracle(keys_np, M - 1, budget_s=args.cpu_budget,
                      max_keys=1 << 24 if n > (1 << 24) else None) if not args.no_cpu else None
    traffic = recorded_traffic(f"{args.workload}:{dom}:{cfg['path']}:{cfg['slice_values']}:{cfg['threads']}")
    line = {
        "metric": METRIC, "value": value, "unit": "Gkeys/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": w["desc"], "n": n, "max_value": M - 1, "keys": w["method"],
                   "l2": f"flushed between timed steps ({args.flush}: 512 MiB write"
                         f"{' + 512 MiB read' if args.flush == 'write+read' else ''}, outside the step events)",
                   "plan": cfg, "wall_s": wall},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "algorithmic_bytes": dom_bytes,
                     "hbm_algorithmic_bytes": dom_hbm_bytes, "hbm_achieved": hbm_achieved,
                     "hbm_frac": hbm_achieved / peak,
                     "kernel_ms": kind_ms[dom], "kernels_ms": kind_ms,
                     "path_achieved": path_achieved, "path_frac": path_achieved / peak,
                     "note": f"dominant kernel '{dom}': frac = its algorithmic bytes by the 8n+M/4 formula "
                             f"(8 B per key, plus M/8 + M/8 bitmap bytes when it builds and reads the bitmap) "
                             f"/ its mean CUDA-event time over {phase_steps} cold-L2 steps; the bucket kernel "
                             f"keeps the M/4 bitmap bytes in shared memory (sparse slices skip most of them), "
                             f"so hbm_frac counts only the bytes it must move through L2/HBM (8n for the "
                             f"bucket and partition kernels); path_frac = 8n+M/4 = {algo_bytes} B / whole-sort "
                             f"step time; peak = {peak_kind} copy bandwidth (MEASURED_PEAKS hbm_gbs)"},
        "e2e": {"value": job_gkeys_s(ws, n, e2e_ms), "unit": "Gkeys/s", "h2d_bytes_per_step": 4 * n,
                "d2h_bytes_per_step": 4 * n + 16, "api": "bitsort_host (pinned host buffers)",
                "overlap": "three streams with a context each; consecutive steps overlap",
                "link": link},
        "gpu_launches": launches,
        "clocks": clk,
        "cpu_baseline": cpu,
        "comparison": comparison,
    }
    print(json.dumps(line), flush=True)


def time_host_link(hbuf, hout, dbuf, stream, reps=10):
    """Host<->device copy rates of this GPU for one step's buffers (pinned
    host memory, copy engines): host-to-device alone, device-to-host alone,
    and both at once on two streams, which is what overlapped steps of the
    end-to-end loop need.  For large arrays the end-to-end loop is bound by
    the both-at-once rate."""
    import torch
    dtmp = torch.empty_like(dbuf)
    other = torch.cuda.Stream()
    nbytes = hbuf.numel() * hbuf.element_size()

    def timed(fn):
        ms = []
        for i in range(reps + 2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            other.wait_event(e0)
            fn()
            done = torch.cuda.Event()
            done.record(other)
            stream.wait_event(done)
            e1.record(stream)
            torch.cuda.synchronize()
            if i >= 2:
                ms.append(e0.elapsed_time(e1))
        return float(np.median(ms))

    def h2d(s):
        with torch.cuda.stream(s):
            dtmp.copy_(hbuf, non_blocking=True)

    def d2h(s):
        with torch.cuda.stream(s):
            hout.copy_(dbuf, non_blocking=True)

    t_h2d = timed(lambda: h2d(stream))
    t_d2h = timed(lambda: d2h(stream))
    t_both = timed(lambda: (h2d(stream), d2h(other)))
    return {"h2d_gbs": nbytes / (t_h2d * 1e-3) / 1e9, "d2h_gbs": nbytes / (t_d2h * 1e-3) / 1e9,
            "duplex_gbs": 2 * nbytes / (t_both * 1e-3) / 1e9,
            "note": "h2d/d2h/duplex: one copy of a step's keys in, out, and both at once (pinned host "
                    "buffers, copy engines, a lone step: latency-bound for small arrays); e2e_gbs: the "
                    "bytes the end-to-end loop moves per step over its step time"}


class L2Flush:
    """Evicts the workload from L2 between timed steps, outside the timed
    events: writes a 512 MiB buffer (larger than the 126 MB L2); mode
    'write+read' then reads a second 512 MiB buffer, so that the L2 holds
    clean lines of an unrelated buffer instead of 512 MiB of dirty flush data
    whose write-back would land inside the next timed step."""

    def __init__(self, mode="write+read"):
        import torch
        self.mode = mode
        self.w = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
        self.r = torch.ones(128 << 20, dtype=torch.float32, device="cuda") if mode == "write+read" else None
        self.sink = torch.zeros(1, dtype=torch.float32, device="cuda")

    def fill_(self, v):
        self.w.fill_(v)
        if self.r is not None:
            self.sink += self.r.sum()


def time_multiset(ctx, keys, M, flush, stream, steps, split_bits, peak):
    """The multiset path (Algorithm 1's stable bit splits, split_bits bits
    per pass; 0 = fewest passes of at most 8 bits) on the same keys: whole
    call time, and the split kernels' bandwidth (8 bytes per key per pass)."""
    import torch
    n = keys.numel()
    out = torch.empty_like(keys)
    res = torch.zeros(2, dtype=torch.int64, device="cuda")
    bits = max(1, (M - 1).bit_length())
    if split_bits:
        d, p = split_bits, -(-bits // split_bits)
    else:
        p = -(-bits // 8)
        d = -(-bits // p)
    ctx.multiset_async(keys, M - 1, split_bits, out=out, result=res, stream=stream)
    torch.cuda.synchronize()
    ok = int(res[0]) & 0xFFFFFFFF == 0 and int(res[1]) == n   # status OK
    ok = ok and bool(torch.all(out[1:].to(torch.int64) & 0xFFFFFFFF >= out[:-1].to(torch.int64) & 0xFFFFFFFF))
    reps = max(3, min(steps, 100))
    ms = []
    for i in range(reps):
        flush.fill_(i & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.multiset_async(keys, M - 1, split_bits, out=out, result=res, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    t = float(np.median(ms))
    ctx.set_phase_timing(True)
    split = []
    for i in range(reps):
        flush.fill_(i & 0xFF)
        ctx.multiset_async(keys, M - 1, split_bits, out=out, result=res, stream=stream)
        torch.cuda.synchronize()
        split.append(dict(ctx.phase_times()).get("msplit", 0.0))
    ctx.set_phase_timing(False)
    per_pass = float(np.median(split)) / p
    gbs = 8 * n / (per_pass * 1e-3) / 1e9 if per_pass > 0 else None
    return {"impl": "bitsort_multiset (Algorithm 1, stable splits)", "split_bits": d, "passes": p, "ms": t,
            "gkeys_s": n / (t * 1e-3) / 1e9, "sorted": ok, "split_ms_per_pass": per_pass,
            "split_gbs": gbs, "split_frac": gbs / peak if gbs else None}


def time_cub(keys, M, flush, stream, steps):
    """cub::DeviceRadixSort::SortKeys on the same keys and GPU (comparison
    point only; a multiset sort on bits [0, ceil(log2 M)))."""
    import ctypes
    import torch
    path = os.path.join(ROOT, "paper_1312_0138_gb300", "compare", "libcubcompare.so")
    if not os.path.exists(path):
        return {"unavailable": "libcubcompare.so not built"}
    lib = ctypes.CDLL(path)
    lib.cub_radix_sort_keys.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int,
                                        ctypes.c_void_p]
    lib.cub_radix_sort_keys.restype = ctypes.c_int
    end_bit = max(1, (M - 1).bit_length())
    out = torch.empty_like(keys)
    n = keys.numel()
    h = stream.cuda_stream
    assert lib.cub_radix_sort_keys(keys.data_ptr(), out.data_ptr(), n, end_bit, h) == 0
    torch.cuda.synchronize()
    reps = max(3, min(steps, 100))
    ms = []
    for i in range(reps):
        flush.fill_(i & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lib.cub_radix_sort_keys(keys.data_ptr(), out.data_ptr(), n, end_bit, h)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    t = float(np.median(ms))
    return {"impl": "cub::DeviceRadixSort::SortKeys", "end_bit": end_bit, "ms": t,
            "gkeys_s": n / (t * 1e-3) / 1e9}


def run_batched(args, ws, rank, local):
    """4096 arrays of uneven sizes and ranges in one persistent launch (graph replay) vs the
    same arrays as 4096 plain launches."""
    import torch
    import gen
    import paper_1312_0138_gb300 as bs

    torch.cuda.set_device(local)
    ctx = bs.Context(local)
    spec = gen.batch_spec(SEED + 3 + 1000 * rank, args.batch_count)
    keys, outs, arrays = [], [], []
    total = 0
    for i, (n, M) in enumerate(spec):
        k = torch.from_numpy(gen.feistel(SEED + 7 * i + 1000 * rank, n, M).view(np.int32)).cuda()
        o = torch.empty_like(k)
        keys.append(k)
        outs.append(o)
        arrays.append((k, M - 1, o))
        total += n
    if args.tune:
        ctx.batch_autotune(arrays)
    plan = ctx.plan(arrays)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        plan.launch()
    res = plan.results()
    bad = [(i, st, cnt) for i, (st, cnt) in enumerate(res) if st != bs.OK or cnt != spec[i][0]]
    assert not bad, f"batched outcomes differ from OK for {len(bad)} arrays, first {bad[:4]}"
    ms = []
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.launch()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    batched_ms = float(np.median(ms))
    # the same arrays as independent plain launches
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.fill_(3)
    e0.record(stream)
    for k, mv, o in arrays:
        ctx.sort_async(k, mv, out=o)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1)
    peak, _ = read_peaks()
    algo = sum(8 * n + M // 4 for n, M in spec)
    line = {"metric": METRIC, "value": total / (batched_ms * 1e-3) / 1e9, "unit": "Gkeys/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": batched_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"batched bitsort, {len(spec)} arrays in one persistent launch (CUDA graph), "
                                   f"n log-uniform [2^10,2^22], max_value log-uniform [2^12,2^26], density [1/64,1/2]",
                       "batch_policy": ctx.get_batch_config(),
                       "total_keys": total, "plain_launches_ms": plain_ms,
                       "plain_launches_gkeys_s": total / (plain_ms * 1e-3) / 1e9,
                       "speedup_vs_plain_launches": plain_ms / batched_ms},
            "roofline": {"bound": "hbm", "achieved": algo / (batched_ms * 1e-3) / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": algo / (batched_ms * 1e-3) / 1e9 / peak, "traffic": None}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_served(args, ws, rank, local):
    """Poisson arrivals of sort requests of uneven sizes through the serving loop."""
    import torch
    import gen
    import paper_1312_0138_gb300 as bs

    torch.cuda.set_device(local)
    count = args.serve_count
    spec = gen.serve_spec(SEED + 4, count, rate_hz=args.rate)
    reqs = []
    for i, (t, n, M) in enumerate(spec):
        k = torch.from_numpy(gen.feistel(SEED + 11 * i, n, M).view(np.int32)).cuda()
        reqs.append((t, k, M - 1, torch.empty_like(k)))
    srv = bs.Server(local, budget_bytes=40 << 30, max_inflight=args.inflight)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tickets = []
    for t, k, mv, o in reqs:
        now = time.perf_counter() - t0
        if t > now:
            time.sleep(t - now)
        tickets.append(srv.submit(k, mv, o))
    lats = []
    for i, tk in enumerate(tickets):
        st, cnt, lat = srv.wait(tk)
        assert st == bs.OK and cnt == spec[i][1], f"request {i} (n={spec[i][1]}, M={spec[i][2]}): status {st}, count {cnt}"
        lats.append(lat)
    wall = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    total = sum(n for _, n, _ in spec)
    # the same requests as one plain call after another (one context, one stream)
    ctx = bs.Context(local)
    for _, k, mv, o in reqs[:3]:
        ctx.sort_async(k, mv, out=o)
    torch.cuda.synchronize()
    p0 = time.perf_counter()
    for _, k, mv, o in reqs:
        ctx.sort_async(k, mv, out=o)
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - p0
    ctx.close()
    line = {"metric": METRIC, "value": total / wall / 1e9, "unit": "Gkeys/s", "n_gpus": ws, "steps": count,
            "warmup": 0, "ms_per_step": wall * 1e3 / count, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"served bitsort, {count} Poisson requests at {args.rate}/s, n log-uniform "
                                   f"[2^10,2^26], max_value log-uniform [2^16,2^32-1], 40 GiB budget",
                       "p50_ms": float(np.percentile(lats, 50)) * 1e3,
                       "p99_ms": float(np.percentile(lats, 99)) * 1e3, "batches": stats["batches"],
                       "max_concurrent_batches": stats["max_concurrent"], "total_keys": total,
                       "plain_calls_s": plain_s, "plain_calls_gkeys_s": total / plain_s / 1e9,
                       "served_over_plain": (total / wall) / (total / plain_s)}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default: 100 for c2a, else 2000)")
    ap.add_argument("--warmup", type=int, default=None, help="warm-up steps (default: 5 for c2a, else 20)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2a", choices=list(WORKLOADS) + ["batched", "served"])
    ap.add_argument("--path", default=None, choices=[None, "fused", "partition", "global"])
    ap.add_argument("--slice", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--wpl", type=int, default=0)
    ap.add_argument("--stage", type=int, default=0)
    ap.add_argument("--layout", type=int, default=1)
    ap.add_argument("--persistent", type=int, default=0)
    ap.add_argument("--emit", type=int, default=0)
    ap.add_argument("--part-stream", type=int, default=0)
    ap.add_argument("--part-threads", type=int, default=0)
    ap.add_argument("--part-tile-keys", type=int, default=0)
    ap.add_argument("--tune", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-cub", action="store_true")
    ap.add_argument("--flush", default="write+read", choices=["write", "write+read"])
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--n-log2", type=int, default=0,
                    help="with --m-log2: a custom plain workload of 2^n-log2 Feistel keys from [0, 2^m-log2) "
                         "(small cases for profiling)")
    ap.add_argument("--m-log2", type=int, default=0)
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--serve-count", type=int, default=400)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--inflight", type=int, default=4)
    args = ap.parse_args()
    if args.n_log2 and args.m_log2:
        n, M = 1 << args.n_log2, 1 << args.m_log2
        assert n <= M
        WORKLOADS["custom"] = dict(n=n, M=M, method="feistel", cfg=5,
                                   desc=f"plain bitsort, one array: n=2^{args.n_log2} distinct uint32 from "
                                        f"[0,2^{args.m_log2}) (Feistel permutation)")
        args.workload = "custom"
    big = args.workload == "c2a"
    if args.steps is None:
        args.steps = 100 if big else 2000
    if args.warmup is None:
        args.warmup = 5 if big else 20
    ws, rank, local = dist_init()
    if args.impl == "reference":
        w = WORKLOADS.get(args.workload, WORKLOADS["c2a"])
        run_reference(args, w, ws, rank)
        return
    if args.workload == "batched":
        run_batched(args, ws, rank, local)
    elif args.workload == "served":
        run_served(args, ws, rank, local)
    else:
        run_plain(args, WORKLOADS[args.workload], ws, rank, local)


if __name__ == "__main__":
    main()
