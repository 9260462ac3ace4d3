"""GB300 (sm_103a) bitmap sort: Python binding of the C ABI in include/bitsort.h.

The operation is the paper's bitwise sort of an integer array (Section V,
Algorithm 1; Theorem 1 fixes the result: the keys in ascending order), done in
its bit-set form on the GPU: every key sets one bit of a bitmap (Table I OR of
a shifted one, Example 2), the set bits are counted (Example 6) and their
positions written out in order (Section II bit numbering).  Keys are distinct
uint32 values bounded by ``max_value``.

This module only marshals arguments: tensors are passed to the CUDA library by
device pointer together with the current torch stream; every step of the sort
runs in the library's kernels.  If ``libbitsort.so`` is missing or cannot be
loaded, importing a function raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Iterable, Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbitsort.so")

OK, ERR_INVALID, ERR_KEY_RANGE, ERR_DUPLICATE, ERR_NOMEM, ERR_TIMEOUT, ERR_CUDA, ERR_BUDGET = range(8)
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "KEY_RANGE", 3: "DUPLICATE", 4: "NOMEM", 5: "TIMEOUT",
                6: "CUDA", 7: "BUDGET"}
PATH_AUTO, PATH_FUSED, PATH_PARTITION, PATH_GLOBAL = range(4)
PATH_NAMES = {0: "auto", 1: "fused", 2: "partition", 3: "global"}

# names every build must export (checked by the CPU test-suite)
EXPORTS = [
    "bitsort_ctx_create", "bitsort_ctx_destroy", "bitsort_status_string", "bitsort_last_error", "bitsort",
    "bitsort_ex", "bitsort_host", "bitsort_i32", "bitsort_multiset", "bitsort_multiset_i32", "bitsort_u16", "bitsort_u8",
    "bitsort_u64",
    "bitsort_sync_status", "bitsort_batched", "bitsort_batch_plan_create", "bitsort_batch_plan_launch",
    "bitsort_batch_plan_results", "bitsort_batch_plan_device_results", "bitsort_batch_plan_destroy",
    "bitsort_server_create", "bitsort_server_submit", "bitsort_server_wait", "bitsort_server_stats",
    "bitsort_server_destroy", "bitsort_autotune", "bitsort_set_config", "bitsort_get_config",
    "bitsort_tune_save", "bitsort_tune_load", "bitsort_set_wait_limit_ms", "bitsort_debug_stalled_launch",
    "bitsort_kernel_launches", "bitsort_noalloc", "bitsort_set_phase_timing", "bitsort_phase_times",
    "bitsort_set_batch_config", "bitsort_get_batch_config", "bitsort_batch_autotune", "bitsort_plan_rule",
    "bitsort_span", "bitsort_range_width", "bitsort_range_split",
]


class BitsortError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)}" if what else STATUS_NAMES.get(status, str(status)))


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("count", ctypes.c_uint64)]


class PlanShape(ctypes.Structure):
    _fields_ = [("slices", ctypes.c_uint32), ("tile_keys", ctypes.c_uint32), ("part_threads", ctypes.c_uint32),
                ("bucket_threads", ctypes.c_uint32), ("smem_bytes", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("scratch_bytes", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class Config(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("slice_values", ctypes.c_uint32), ("block_threads", ctypes.c_uint32),
                ("words_per_lane", ctypes.c_uint32), ("stage", ctypes.c_uint32), ("layout", ctypes.c_uint32),
                ("persistent", ctypes.c_uint32), ("emit", ctypes.c_uint32), ("part_stream", ctypes.c_uint32),
                ("summary", ctypes.c_uint32), ("part_threads", ctypes.c_uint32),
                ("part_tile_keys", ctypes.c_uint32), ("ms", ctypes.c_double)]

    def as_dict(self):
        return {"path": PATH_NAMES.get(self.path, self.path), "slice_values": self.slice_values,
                "threads": self.block_threads, "words_per_lane": self.words_per_lane, "stage": self.stage,
                "layout": LAYOUT_NAMES.get(self.layout, self.layout), "persistent": self.persistent,
                "emit": EMIT_NAMES.get(self.emit, self.emit), "part_stream": self.part_stream,
                "summary": self.summary, "part_threads": self.part_threads,
                "part_tile_keys": self.part_tile_keys, "ms": self.ms}


LAYOUT_EXACT, LAYOUT_CAPACITY = 0, 1
LAYOUT_NAMES = {0: "exact", 1: "capacity"}
EMIT_WORD, EMIT_RANK = 0, 1
EMIT_NAMES = {0: "word", 1: "rank"}


class Desc(ctypes.Structure):
    _fields_ = [("keys", ctypes.c_void_p), ("out", ctypes.c_void_p), ("n", ctypes.c_uint64),
                ("max_value", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    from . import builder as _b
    return _b.build(force=force)


def _declare(lib):
    p, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    st = ctypes.c_int
    sig = {
        "bitsort_ctx_create": (st, [i32, ctypes.POINTER(p)]),
        "bitsort_ctx_destroy": (st, [p]),
        "bitsort_status_string": (ctypes.c_char_p, [i32]),
        "bitsort_last_error": (ctypes.c_char_p, []),
        "bitsort": (st, [p, ctypes.c_size_t, u32, p, p]),
        "bitsort_ex": (st, [p, p, u64, u32, p, p, p]),
        "bitsort_i32": (st, [p, p, u64, ctypes.c_int32, ctypes.c_int32, p, p, p]),
        "bitsort_span": (st, [p, p, u64, u32, u32, p, p, p]),
        "bitsort_range_width": (u64, [u32, u32]),
        "bitsort_range_split": (st, [p, p, u64, u32, u32, p, p, p, p]),
        "bitsort_host": (st, [p, p, u64, u32, p, p, p]),
        "bitsort_multiset": (st, [p, p, u64, u32, u32, p, p, p]),
        "bitsort_u16": (st, [p, p, u64, ctypes.c_uint16, p, p, p]),
        "bitsort_u8": (st, [p, p, u64, ctypes.c_uint8, p, p, p]),
        "bitsort_u64": (st, [p, p, u64, u64, p, p, p]),
        "bitsort_multiset_i32": (st, [p, p, u64, ctypes.c_int32, ctypes.c_int32, u32, p, p, p]),
        "bitsort_sync_status": (st, [p, p, ctypes.POINTER(u64)]),
        "bitsort_batched": (st, [p, p, ctypes.c_size_t, p, p]),
        "bitsort_batch_plan_create": (st, [p, p, ctypes.c_size_t, ctypes.POINTER(p)]),
        "bitsort_batch_plan_launch": (st, [p, p]),
        "bitsort_batch_plan_results": (st, [p, p, p]),
        "bitsort_batch_plan_device_results": (p, [p]),
        "bitsort_batch_plan_destroy": (st, [p]),
        "bitsort_server_create": (st, [i32, u64, i32, ctypes.POINTER(p)]),
        "bitsort_server_submit": (st, [p, p, u64, u32, p, ctypes.POINTER(u64)]),
        "bitsort_server_wait": (st, [p, u64, ctypes.POINTER(i32), ctypes.POINTER(u64),
                                     ctypes.POINTER(ctypes.c_double)]),
        "bitsort_server_stats": (st, [p] + [ctypes.POINTER(u64)] * 4),
        "bitsort_server_destroy": (st, [p]),
        "bitsort_autotune": (st, [p, p, p, u64, u32, ctypes.POINTER(Config)]),
        "bitsort_set_config": (st, [p, u64, u32, ctypes.POINTER(Config)]),
        "bitsort_get_config": (st, [p, u64, u32, ctypes.POINTER(Config)]),
        "bitsort_plan_rule": (st, [i32, u32, u64, u32, ctypes.POINTER(Config), ctypes.POINTER(PlanShape)]),
        "bitsort_tune_save": (st, [p, ctypes.c_char_p]),
        "bitsort_tune_load": (st, [p, ctypes.c_char_p]),
        "bitsort_set_wait_limit_ms": (st, [p, u32]),
        "bitsort_debug_stalled_launch": (st, [p, p, u64, u32, p, p]),
        "bitsort_kernel_launches": (u64, [p]),
        "bitsort_noalloc": (st, [p, u64, u32, p, p, p]),
        "bitsort_set_phase_timing": (st, [p, i32]),
        "bitsort_set_batch_config": (st, [p, ctypes.POINTER(Config)]),
        "bitsort_get_batch_config": (st, [p, ctypes.POINTER(Config)]),
        "bitsort_batch_autotune": (st, [p, p, ctypes.c_size_t, ctypes.POINTER(Config)]),
        "bitsort_phase_times": (st, [p, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(i32),
                                     ctypes.POINTER(i32)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def load(path: Optional[str] = None):
    """Load libbitsort.so (raises if it was not built: no fallback path)."""
    global _lib
    with _lock:
        if _lib is None:
            path = path or LIB_PATH
            if not os.path.exists(path):
                raise ImportError(f"libbitsort.so not built ({path}); run __graft_entry__.build()")
            _lib = _declare(ctypes.CDLL(path))
    return _lib


def _check(status: int, what: str):
    if status != OK:
        detail = ""
        if status in (ERR_CUDA, ERR_NOMEM) and _lib is not None:
            detail = " [" + (_lib.bitsort_last_error() or b"").decode(errors="replace") + "]"
        raise BitsortError(status, what + detail)


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t, dtypes=None) -> int:
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda:
        raise ValueError("tensor must be on a CUDA device")
    if t.dtype not in (dtypes or (torch.int32, torch.uint32)):
        raise TypeError(f"keys/out of type {t.dtype}: expected one of {dtypes or (torch.int32, torch.uint32)}")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _host_ptr(t, allow_int64: bool = False) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError("expected a CPU tensor")
    ok = (torch.int32, torch.uint32) + ((torch.int64,) if allow_int64 else ())
    if t.dtype not in ok or not t.is_contiguous():
        raise TypeError(f"host tensor of type {t.dtype}: expected a contiguous tensor of {ok}")
    return t.data_ptr()


class Context:
    """A bitsort context on one device: scratch, tuned table, launch counter."""

    def __init__(self, device: int = 0):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.bitsort_ctx_create(device, ctypes.byref(h)), "bitsort_ctx_create")
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            load().bitsort_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # single sort -----------------------------------------------------------
    def sort_async(self, keys, max_value: int, out=None, result=None, stream=None):
        """Enqueue the sort of `keys` (device tensor) into `out`; returns out.

        `result` is an optional device tensor of 2 int64 (bitsort_result_t)."""
        import torch
        if out is None:
            out = torch.empty_like(keys)
        rptr = result.data_ptr() if result is not None else None
        st = load().bitsort_ex(self.handle, _ptr(keys) if keys.numel() else None, keys.numel(),
                               int(max_value), _ptr(out) if out.numel() else None, rptr, _stream_handle(stream))
        _check(st, "bitsort_ex")
        return out

    def sort_i32_async(self, keys, min_value: int, max_value: int, out=None, result=None, stream=None):
        """Enqueue the sort of signed int32 `keys` in [min_value, max_value]; returns out."""
        import torch
        if out is None:
            out = torch.empty_like(keys)
        rptr = result.data_ptr() if result is not None else None
        st = load().bitsort_i32(self.handle, _ptr(keys) if keys.numel() else None, keys.numel(), int(min_value),
                                int(max_value), _ptr(out) if out.numel() else None, rptr, _stream_handle(stream))
        _check(st, "bitsort_i32")
        return out

    def sort_i32(self, keys, min_value: int, max_value: int, out=None, stream=None):
        """Signed sort and wait: returns (status, count, out)."""
        out = self.sort_i32_async(keys, min_value, max_value, out=out, stream=stream)
        st, cnt = self.sync_status(stream)
        return st, cnt, out

    def sort_span_async(self, keys, min_value: int, max_value: int, out=None, result=None, stream=None):
        """Enqueue the sort of distinct uint32 `keys` in [min_value, max_value]
        (C entry point bitsort_span); returns out."""
        import torch
        if out is None:
            out = torch.empty_like(keys)
        rptr = result.data_ptr() if result is not None else None
        st = load().bitsort_span(self.handle, _ptr(keys) if keys.numel() else None, keys.numel(), int(min_value),
                                 int(max_value), _ptr(out) if out.numel() else None, rptr, _stream_handle(stream))
        _check(st, "bitsort_span")
        return out

    def range_split_async(self, keys, max_value: int, parts: int, out=None, counts=None, result=None,
                          stream=None):
        """Enqueue the grouping of `keys` by the rank that owns their value
        range (C entry point bitsort_range_split); returns (out, counts), counts
        a device int64 tensor of `parts` group sizes."""
        import torch
        if out is None:
            out = torch.empty_like(keys)
        if counts is None:
            counts = torch.empty(parts, dtype=torch.int64, device=keys.device)
        rptr = result.data_ptr() if result is not None else None
        st = load().bitsort_range_split(self.handle, _ptr(keys) if keys.numel() else None, keys.numel(),
                                        int(max_value), int(parts), _ptr(out) if out.numel() else None,
                                        _ptr(counts, (torch.int64,)), rptr, _stream_handle(stream))
        _check(st, "bitsort_range_split")
        return out, counts

    def sort_width_async(self, keys, max_value: int, out=None, result=None, stream=None):
        """Bitmap sort of 16-, 8- or 64-bit keys (torch int16 / uint8 / int64
        tensors holding the unsigned values); returns out."""
        import torch
        fn = {torch.int16: "bitsort_u16", torch.uint8: "bitsort_u8", torch.int64: "bitsort_u64"}.get(keys.dtype)
        if fn is None:
            raise TypeError(f"no bitmap sort for keys of type {keys.dtype}")
        if out is None:
            out = torch.empty_like(keys)
        rptr = result.data_ptr() if result is not None else None
        dt = (keys.dtype,)
        st = getattr(load(), fn)(self.handle, _ptr(keys, dt) if keys.numel() else None, keys.numel(),
                                 int(max_value), _ptr(out, dt) if out.numel() else None, rptr,
                                 _stream_handle(stream))
        _check(st, fn)
        return out

    def sort_width(self, keys, max_value: int, out=None, stream=None):
        """Width sort and wait: returns (status, count, out)."""
        out = self.sort_width_async(keys, max_value, out=out, stream=stream)
        st, cnt = self.sync_status(stream)
        return st, cnt, out

    def multiset_async(self, keys, max_value: int, split_bits: int = 0, out=None, result=None, stream=None):
        """Enqueue Algorithm 1 (stable bit splits; keys may repeat) on `keys`; returns out."""
        import torch
        if out is None:
            out = torch.empty_like(keys)
        rptr = result.data_ptr() if result is not None else None
        st = load().bitsort_multiset(self.handle, _ptr(keys) if keys.numel() else None, keys.numel(),
                                     int(max_value), int(split_bits), _ptr(out) if out.numel() else None, rptr,
                                     _stream_handle(stream))
        _check(st, "bitsort_multiset")
        return out

    def multiset(self, keys, max_value: int, split_bits: int = 0, out=None, stream=None):
        """Multiset sort and wait: returns (status, count, out)."""
        out = self.multiset_async(keys, max_value, split_bits, out=out, stream=stream)
        st, cnt = self.sync_status(stream)
        return st, cnt, out

    def multiset_i32_async(self, keys, min_value: int, max_value: int, split_bits: int = 0, out=None,
                           result=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(keys)
        rptr = result.data_ptr() if result is not None else None
        st = load().bitsort_multiset_i32(self.handle, _ptr(keys) if keys.numel() else None, keys.numel(),
                                         int(min_value), int(max_value), int(split_bits),
                                         _ptr(out) if out.numel() else None, rptr, _stream_handle(stream))
        _check(st, "bitsort_multiset_i32")
        return out

    def multiset_i32(self, keys, min_value: int, max_value: int, split_bits: int = 0, out=None, stream=None):
        out = self.multiset_i32_async(keys, min_value, max_value, split_bits, out=out, stream=stream)
        st, cnt = self.sync_status(stream)
        return st, cnt, out

    def sort_host_async(self, h_keys, max_value: int, h_out, h_result=None, stream=None):
        """Enqueue the sort of HOST keys (CPU int32/uint32 tensor, page-locked
        for asynchronous copies) into the HOST tensor h_out through the C
        entry point `bitsort_host`; h_result (CPU int64 tensor of 2) receives
        (status, count) once the stream passes the call."""
        _check(load().bitsort_host(self.handle, _host_ptr(h_keys) if h_keys.numel() else None, h_keys.numel(),
                                   int(max_value), _host_ptr(h_out) if h_out.numel() else None,
                                   _host_ptr(h_result, allow_int64=True) if h_result is not None else None,
                                   _stream_handle(stream)), "bitsort_host")
        return h_out

    def sync_status(self, stream=None):
        cnt = ctypes.c_uint64(0)
        st = load().bitsort_sync_status(self.handle, _stream_handle(stream), ctypes.byref(cnt))
        return st, cnt.value

    def sort(self, keys, max_value: int, out=None, stream=None):
        """Sort and wait: returns (status, count, out)."""
        out = self.sort_async(keys, max_value, out=out, stream=stream)
        st, cnt = self.sync_status(stream)
        return st, cnt, out

    # tuning ----------------------------------------------------------------
    def set_config(self, n: int, max_value: int, path: int, slice_values: int = 0, threads: int = 0,
                   words_per_lane: int = 0, stage: int = 0, layout: int = LAYOUT_CAPACITY, persistent: int = 0,
                   emit: int = EMIT_WORD, part_stream: int = 0, summary: int = 1, part_threads: int = 0,
                   part_tile_keys: int = 0):
        cfg = Config(path, slice_values, threads, words_per_lane, stage, layout, persistent, emit, part_stream,
                     summary, part_threads, part_tile_keys, 0.0)
        _check(load().bitsort_set_config(self.handle, n, max_value, ctypes.byref(cfg)), "bitsort_set_config")

    def get_config(self, n: int, max_value: int):
        cfg = Config()
        _check(load().bitsort_get_config(self.handle, n, max_value, ctypes.byref(cfg)), "bitsort_get_config")
        return cfg.as_dict()

    def autotune(self, keys, max_value: int, out=None):
        import torch
        if out is None:
            out = torch.empty_like(keys)
        cfg = Config()
        _check(load().bitsort_autotune(self.handle, _ptr(keys), _ptr(out), keys.numel(), int(max_value),
                                       ctypes.byref(cfg)), "bitsort_autotune")
        return cfg.as_dict()

    def tune_save(self, path: str):
        _check(load().bitsort_tune_save(self.handle, path.encode()), "bitsort_tune_save")

    def tune_load(self, path: str):
        _check(load().bitsort_tune_load(self.handle, path.encode()), "bitsort_tune_load")

    def set_wait_limit_ms(self, ms: int):
        _check(load().bitsort_set_wait_limit_ms(self.handle, ms), "bitsort_set_wait_limit_ms")

    def debug_stalled_launch(self, keys, max_value: int, out, stream=None):
        _check(load().bitsort_debug_stalled_launch(self.handle, _ptr(keys), keys.numel(), int(max_value),
                                                   _ptr(out), _stream_handle(stream)), "debug_stalled_launch")

    def set_phase_timing(self, enable: bool):
        _check(load().bitsort_set_phase_timing(self.handle, 1 if enable else 0), "bitsort_set_phase_timing")

    def phase_times(self):
        """[(kind, ms), ...] of the last single sort's kernels (phase timing on)."""
        ms = (ctypes.c_float * 8)()
        kinds = (ctypes.c_int * 8)()
        cnt = ctypes.c_int(0)
        _check(load().bitsort_phase_times(self.handle, ms, kinds, ctypes.byref(cnt)), "bitsort_phase_times")
        names = {-1: "persistent", 0: "hist", 1: "part", 2: "bucket", 3: "gscatter", 4: "gscan", 5: "parts",
                 6: "partw", 16: "mhist", 17: "msplit"}
        return [(names.get(kinds[i], kinds[i]), ms[i]) for i in range(cnt.value)]

    def kernel_launches(self) -> int:
        return int(load().bitsort_kernel_launches(self.handle))

    # batching --------------------------------------------------------------
    def batched(self, arrays: Sequence, results=None, stream=None):
        """Sort [(keys, max_value, out), ...] in one launch; `results` is an
        optional device tensor of len(arrays) x 2 int64 outcomes."""
        descs = _descs(arrays)
        rptr = results.data_ptr() if results is not None else None
        _check(load().bitsort_batched(self.handle, ctypes.byref(descs), len(arrays), rptr,
                                      _stream_handle(stream)), "bitsort_batched")

    def plan(self, arrays: Sequence) -> "BatchPlan":
        return BatchPlan(self, arrays)

    def set_batch_config(self, path: int = PATH_PARTITION, slice_values: int = 0, threads: int = 0,
                         words_per_lane: int = 0, stage: int = 0):
        cfg = Config(path, slice_values, threads, words_per_lane, stage, 0, 1, 0, 0, 1, 0, 0, 0.0)
        _check(load().bitsort_set_batch_config(self.handle, ctypes.byref(cfg)), "bitsort_set_batch_config")

    def get_batch_config(self):
        cfg = Config()
        _check(load().bitsort_get_batch_config(self.handle, ctypes.byref(cfg)), "bitsort_get_batch_config")
        return cfg.as_dict()

    def batch_autotune(self, arrays: Sequence):
        descs = _descs(arrays)
        cfg = Config()
        _check(load().bitsort_batch_autotune(self.handle, ctypes.byref(descs), len(arrays), ctypes.byref(cfg)),
               "bitsort_batch_autotune")
        return cfg.as_dict()


def _descs(arrays):
    descs = (Desc * len(arrays))()
    for i, (keys, max_value, out) in enumerate(arrays):
        descs[i].keys = _ptr(keys) if keys.numel() else None
        descs[i].out = _ptr(out) if out.numel() else None
        descs[i].n = keys.numel()
        descs[i].max_value = int(max_value)
    return descs


class BatchPlan:
    """A reusable batched sort (one persistent launch, replayed from a CUDA graph)."""

    def __init__(self, ctx: Context, arrays: Sequence):
        self.ctx = ctx
        self.count = len(arrays)
        self._keep = list(arrays)
        h = ctypes.c_void_p()
        descs = _descs(arrays)
        _check(load().bitsort_batch_plan_create(ctx.handle, ctypes.byref(descs), self.count, ctypes.byref(h)),
               "bitsort_batch_plan_create")
        self.handle = h

    def launch(self, stream=None):
        _check(load().bitsort_batch_plan_launch(self.handle, _stream_handle(stream)), "bitsort_batch_plan_launch")

    def results(self, stream=None):
        res = (Result * self.count)()
        load().bitsort_batch_plan_results(self.handle, _stream_handle(stream), ctypes.byref(res))
        return [(r.status, r.count) for r in res]

    def close(self):
        if self.handle:
            load().bitsort_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching sort server (admission by a device-memory budget)."""

    def __init__(self, device: int = 0, budget_bytes: int = 40 << 30, max_inflight: int = 4):
        h = ctypes.c_void_p()
        _check(load().bitsort_server_create(device, budget_bytes, max_inflight, ctypes.byref(h)),
               "bitsort_server_create")
        self.handle = h
        self._keep = {}

    def submit(self, keys, max_value: int, out) -> int:
        t = ctypes.c_uint64(0)
        _check(load().bitsort_server_submit(self.handle, _ptr(keys) if keys.numel() else None, keys.numel(),
                                            int(max_value), _ptr(out) if out.numel() else None, ctypes.byref(t)),
               "bitsort_server_submit")
        self._keep[t.value] = (keys, out)
        return t.value

    def wait(self, ticket: int):
        st, cnt, lat = ctypes.c_int(0), ctypes.c_uint64(0), ctypes.c_double(0)
        load().bitsort_server_wait(self.handle, ticket, ctypes.byref(st), ctypes.byref(cnt), ctypes.byref(lat))
        self._keep.pop(ticket, None)
        return st.value, cnt.value, lat.value

    def stats(self):
        v = [ctypes.c_uint64(0) for _ in range(4)]
        load().bitsort_server_stats(self.handle, *[ctypes.byref(x) for x in v])
        return {"completed": v[0].value, "keys": v[1].value, "batches": v[2].value,
                "max_concurrent": v[3].value}

    def close(self):
        if self.handle:
            load().bitsort_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default_ctx = {}


def default_context(device: Optional[int] = None) -> Context:
    import torch
    dev = torch.cuda.current_device() if device is None else device
    if dev not in _default_ctx:
        _default_ctx[dev] = Context(dev)
    return _default_ctx[dev]


def bitsort(keys, max_value: int, out=None, stream=None):
    """The plain call: enqueue the sort of `keys` into `out` on `stream`
    (default: torch's current stream) through the C entry point `bitsort`
    (per-device default context); returns `out`.  Host-checkable errors raise
    BitsortError; read the data-dependent status with :func:`sync_status`."""
    import torch
    if out is None:
        out = torch.empty_like(keys)
    st = load().bitsort(_ptr(keys) if keys.numel() else None, keys.numel(), int(max_value),
                        _ptr(out) if out.numel() else None, _stream_handle(stream))
    _check(st, "bitsort")
    return out


def bitsort_i32(keys, min_value: int, max_value: int, out=None, stream=None):
    """Enqueue the sort of signed int32 `keys` in [min_value, max_value]
    through the C entry point `bitsort_i32` (per-device default context);
    returns `out`.  Read the status with :func:`sync_status`."""
    return default_context(keys.device.index).sort_i32_async(keys, min_value, max_value, out=out, stream=stream)


def bitsort_noalloc(keys, max_value: int, out, result, stream=None):
    """Enqueue the sort through the C entry point `bitsort_noalloc`, which
    allocates no device memory: `out` must not overlap `keys`, `result` is a
    device tensor of 2 int64 receiving (status, count)."""
    st = load().bitsort_noalloc(_ptr(keys) if keys.numel() else None, keys.numel(), int(max_value),
                                _ptr(out) if out.numel() else None, result.data_ptr(), _stream_handle(stream))
    _check(st, "bitsort_noalloc")
    return out


def range_width(max_value: int, parts: int) -> int:
    """Values per rank of a sort spread over `parts` ranks by value range
    (C entry point bitsort_range_width)."""
    return int(load().bitsort_range_width(int(max_value), int(parts)))


def sync_status(stream=None):
    """Status and count of the last plain `bitsort` call (waits for `stream`)."""
    cnt = ctypes.c_uint64(0)
    st = load().bitsort_sync_status(None, _stream_handle(stream), ctypes.byref(cnt))
    return st, cnt.value


def plan_rule(sms: int, smem_per_block: int, n: int, max_value: int):
    """The built-in plan for n distinct keys bounded by max_value on a device
    with `sms` SMs and `smem_per_block` bytes of opt-in shared memory per
    block, through the C entry point `bitsort_plan_rule` (host logic only: no
    GPU needed).  Returns (configuration dict, shape dict)."""
    cfg, shape = Config(), PlanShape()
    _check(load().bitsort_plan_rule(int(sms), int(smem_per_block), int(n), int(max_value), ctypes.byref(cfg),
                                    ctypes.byref(shape)), "bitsort_plan_rule")
    return cfg.as_dict(), shape.as_dict()
