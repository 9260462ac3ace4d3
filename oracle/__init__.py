"""CPU oracle for the bitwise sort -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline / reference leg may import this package.  The GPU library
(``paper_1312_0138_gb300``) never imports it and shares no code with it.

Thin ctypes wrapper over ``oracle.c`` (plain C, compiled with gcc on first
use).  See ``oracle.c`` for the passage of the paper each function restates.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, KEY_RANGE, DUPLICATE, NOMEM = 0, 2, 3, 4


def compile_library(source: str, out_path: str) -> str:
    """gcc -O2 -shared of one C file (also used by tests that build mutants)."""
    tmp = out_path + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, source])
    os.replace(tmp, out_path)
    return out_path


def build(force: bool = False) -> str:
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(SOURCE)):
        return _LIB_PATH
    return compile_library(SOURCE, _LIB_PATH)


def bind(path: str):
    """Load an oracle library and declare its signatures."""
    lib = ctypes.CDLL(path)
    u64, p, u32 = ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint32
    lib.oracle_bit_value.argtypes = [u32, ctypes.c_uint]
    lib.oracle_bit_value.restype = ctypes.c_int
    lib.oracle_bit_or.argtypes = [u32, u32]
    lib.oracle_bit_or.restype = u32
    lib.oracle_bin_repl_i16.argtypes = [ctypes.c_int16, ctypes.c_char_p]
    lib.oracle_bin_repl_i16.restype = None
    lib.oracle_bitmap_sort.argtypes = [p, u64, u32, p, ctypes.POINTER(u64)]
    lib.oracle_bitmap_sort.restype = ctypes.c_int
    lib.oracle_paper_sort_u32.argtypes = [p, u64, ctypes.c_int]
    lib.oracle_paper_sort_u32.restype = ctypes.c_int
    lib.oracle_paper_sort_i32.argtypes = [p, u64]
    lib.oracle_paper_sort_i32.restype = ctypes.c_int
    lib.oracle_bitmap_sort_i32.argtypes = [p, u64, ctypes.c_int32, ctypes.c_int32, p,
                                           ctypes.POINTER(u64)]
    lib.oracle_bitmap_sort_i32.restype = ctypes.c_int
    lib.oracle_bitmap_sort_u64.argtypes = [p, u64, u64, p, ctypes.POINTER(u64)]
    lib.oracle_bitmap_sort_u64.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = bind(build())
    return _lib


class Oracle:
    """Python face of one loaded oracle library (the real one, or a mutant
    built by a test)."""

    def __init__(self, lib=None):
        self.lib = lib if lib is not None else _load()

    def bit_value(self, x: int, i: int) -> int:
        return self.lib.oracle_bit_value(x, i)

    def bit_or(self, x: int, y: int) -> int:
        return self.lib.oracle_bit_or(x, y)

    def bin_repl_i16(self, v: int) -> str:
        buf = ctypes.create_string_buffer(17)
        self.lib.oracle_bin_repl_i16(v, buf)
        return buf.value.decode()

    def bitmap_sort(self, keys, max_value: int):
        """(status, sorted distinct in-range keys) -- the bitmap sort."""
        keys = np.ascontiguousarray(keys, dtype=np.uint32)
        out = np.empty(max(keys.size, 1), dtype=np.uint32)
        count = ctypes.c_uint64(0)
        st = self.lib.oracle_bitmap_sort(keys.ctypes.data, keys.size, int(max_value),
                                         out.ctypes.data, ctypes.byref(count))
        if st == NOMEM:
            raise MemoryError("oracle bitmap allocation failed")
        return st, out[:count.value].copy()

    def paper_sort_u32(self, keys, nbits: int = 32) -> np.ndarray:
        """Algorithm 1 (stable one-bit splits, bits 0..nbits-1) on a copy."""
        a = np.array(keys, dtype=np.uint32, copy=True)
        if self.lib.oracle_paper_sort_u32(a.ctypes.data, a.size, nbits) != 0:
            raise MemoryError("oracle_paper_sort_u32 failed")
        return a

    def paper_sort_i32(self, keys) -> np.ndarray:
        """Algorithm 1 with its sign split, for int32 keys, on a copy."""
        a = np.array(keys, dtype=np.int32, copy=True)
        if self.lib.oracle_paper_sort_i32(a.ctypes.data, a.size) != 0:
            raise MemoryError("oracle_paper_sort_i32 failed")
        return a

    def bitmap_sort_i32(self, keys, min_value: int, max_value: int):
        keys = np.ascontiguousarray(keys, dtype=np.int32)
        out = np.empty(max(keys.size, 1), dtype=np.int32)
        count = ctypes.c_uint64(0)
        st = self.lib.oracle_bitmap_sort_i32(keys.ctypes.data, keys.size, int(min_value),
                                             int(max_value), out.ctypes.data, ctypes.byref(count))
        if st < 0 or st == NOMEM:
            raise ValueError("oracle_bitmap_sort_i32 failed")
        return st, out[:count.value].copy()

    def bitmap_sort_u64(self, keys, max_value: int):
        """Bitmap sort of 64-bit keys bounded by max_value (< 2^40)."""
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        out = np.empty(max(keys.size, 1), dtype=np.uint64)
        count = ctypes.c_uint64(0)
        st = self.lib.oracle_bitmap_sort_u64(keys.ctypes.data, keys.size, int(max_value), out.ctypes.data,
                                             ctypes.byref(count))
        if st < 0 or st == NOMEM:
            raise ValueError("oracle_bitmap_sort_u64 failed")
        return st, out[:count.value].copy()

    def batched(self, arrays):
        """Bitmap sort of each (keys, max_value) pair, one after another."""
        return [self.bitmap_sort(k, mv) for k, mv in arrays]


_default = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle()
    return _default


def bitmap_sort(keys, max_value: int):
    return default().bitmap_sort(keys, max_value)


def paper_sort_u32(keys, nbits: int = 32):
    return default().paper_sort_u32(keys, nbits)


def paper_sort_i32(keys):
    return default().paper_sort_i32(keys)


def batched(arrays):
    return default().batched(arrays)
