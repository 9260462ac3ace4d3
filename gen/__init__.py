"""Seeded synthetic inputs for the bitmap sort (shared by the oracle's tests,
the GPU tests and the benchmark).

Holds only random sampling: Floyd sampling + Fisher-Yates shuffles, a keyed
Feistel bijection of [0, M) with cycle walking, uniform draws with
replacement, and the log-uniform / Poisson recipes of the batched and served
workloads.  The C source (``gen.c``) names the published definition of each
generator.  Nothing here sorts, sets bits or counts bits.

Workload recipes (sizes of the paper's problem: sort an integer array,
Algorithm 1, Theorem 1; keys distinct and bounded by ``max_value`` because the
bitmap form of the method needs both):

* ``floyd``   -- n distinct keys uniform without replacement from [0, M).
* ``feistel`` -- keys[i] = pi(i), i < n, pi a pseudo-random bijection of [0, M):
  n distinct keys in random order; O(n) and parallel, used where Floyd's
  sequential sampling would take minutes (n = 2^31).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB_PATH = os.path.join(_HERE, "libgen.so")
_lock = threading.Lock()
_lib = None

SEED_BASE = 0x13120138


def build(force: bool = False) -> str:
    """Compile gen.c into libgen.so beside it (gcc, -O2, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, p = ctypes.c_uint64, ctypes.c_void_p
            lib.gen_floyd_shuffled.argtypes = [u64, u64, u64, p]
            lib.gen_floyd_shuffled.restype = ctypes.c_int
            lib.gen_shuffle_u32.argtypes = [u64, p, u64]
            lib.gen_shuffle_u32.restype = None
            lib.gen_uniform_u32.argtypes = [u64, u64, u64, p]
            lib.gen_uniform_u32.restype = ctypes.c_int
            lib.gen_unit_f64.argtypes = [u64, u64, p]
            lib.gen_unit_f64.restype = None
            lib.gen_feistel_perm.argtypes = [u64, u64, u64, u64, p]
            lib.gen_feistel_perm.restype = ctypes.c_int
            lib.gen_feistel_inverse.argtypes = [u64, u64, p, u64, p]
            lib.gen_feistel_inverse.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def floyd(seed: int, n: int, M: int) -> np.ndarray:
    """n distinct uint32 keys uniform without replacement from [0, M), shuffled."""
    if n > M:
        raise ValueError("n > M: keys cannot be distinct")
    out = np.empty(n, dtype=np.uint32)
    if n:
        rc = _load().gen_floyd_shuffled(seed, n, M, _ptr(out))
        if rc != 0:
            raise RuntimeError(f"gen_floyd_shuffled failed ({rc})")
    return out


def feistel(seed: int, n: int, M: int, start: int = 0, out: np.ndarray | None = None) -> np.ndarray:
    """keys[i] = pi(start + i) for i < n; pi a seeded bijection of [0, M)."""
    if start + n > M:
        raise ValueError("start + n > M")
    if out is None:
        out = np.empty(n, dtype=np.uint32)
    assert out.dtype == np.uint32 and out.flags.c_contiguous and out.size == n
    if n:
        rc = _load().gen_feistel_perm(seed, M, start, n, _ptr(out))
        if rc != 0:
            raise RuntimeError(f"gen_feistel_perm failed ({rc})")
    return out


def feistel_inverse(seed: int, M: int, y: np.ndarray) -> np.ndarray:
    """pi^{-1}(y) for the bijection used by :func:`feistel` (uint64 result)."""
    y = np.ascontiguousarray(y, dtype=np.uint32)
    out = np.empty(y.size, dtype=np.uint64)
    if y.size:
        rc = _load().gen_feistel_inverse(seed, M, _ptr(y), y.size, _ptr(out))
        if rc != 0:
            raise RuntimeError("gen_feistel_inverse failed")
    return out


def shuffle(seed: int, a: np.ndarray) -> np.ndarray:
    """Seeded Fisher-Yates shuffle of a copy of ``a`` (uint32)."""
    b = np.array(a, dtype=np.uint32, copy=True)
    _load().gen_shuffle_u32(seed, _ptr(b), b.size)
    return b


def uniform_with_replacement(seed: int, n: int, M: int) -> np.ndarray:
    """n uniform draws from [0, M) with replacement (duplicates allowed)."""
    out = np.empty(n, dtype=np.uint32)
    if n:
        if _load().gen_uniform_u32(seed, n, M, _ptr(out)) != 0:
            raise RuntimeError("gen_uniform_u32 failed")
    return out


def unit(seed: int, count: int) -> np.ndarray:
    """count uniform doubles in [0, 1)."""
    out = np.empty(count, dtype=np.float64)
    if count:
        _load().gen_unit_f64(seed, count, _ptr(out))
    return out


def keys(seed: int, n: int, M: int, method: str = "auto") -> np.ndarray:
    """Distinct keys by the named recipe ('floyd', 'feistel' or 'auto':
    Floyd up to 2^25 keys, Feistel beyond)."""
    if method == "auto":
        method = "floyd" if n <= (1 << 25) else "feistel"
    if method == "floyd":
        return floyd(seed, n, M)
    if method == "feistel":
        return feistel(seed, n, M)
    raise ValueError(method)


# ---------------------------------------------------------------- workloads
def log_uniform_int(u: float, lo: float, hi: float) -> int:
    """exp(ln lo + u (ln hi - ln lo)) rounded down, clamped to [lo, hi]."""
    v = int(math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo))))
    return max(int(lo), min(int(hi), v))


def batch_spec(seed: int, count: int = 4096, n_lo: int = 1 << 10, n_hi: int = 1 << 22,
               m_lo: int = 1 << 12, m_hi: int = 1 << 26,
               dens_lo: float = 1 / 64, dens_hi: float = 1 / 2):
    """Per-array (n_i, M_i) of the batched workload.

    n_i log-uniform in [n_lo, n_hi]; M_i log-uniform in
    [max(m_lo, n_i/dens_hi), min(m_hi, n_i/dens_lo)] (never empty for the
    default bounds), so max_value_i = M_i - 1 lies in [m_lo - 1, m_hi - 1]
    and the density n_i/M_i in [dens_lo, dens_hi] wherever the range bounds
    allow it.
    """
    u = unit(seed, 2 * count)
    spec = []
    for i in range(count):
        n = log_uniform_int(u[2 * i], n_lo, n_hi)
        lo = max(m_lo, int(math.ceil(n / dens_hi)))
        hi = min(m_hi, int(n / dens_lo))
        if hi < lo:
            hi = lo
        M = log_uniform_int(u[2 * i + 1], lo, hi)
        spec.append((n, M))
    return spec


def serve_spec(seed: int, count: int, rate_hz: float, n_lo: int = 1 << 10, n_hi: int = 1 << 26,
               m_lo: int = 1 << 16, m_hi: int = (1 << 32)):
    """Poisson request stream of the served workload: (arrival_s, n, M) triples.

    Gaps are exponential with mean 1/rate_hz; M log-uniform in [m_lo, m_hi];
    n log-uniform in [n_lo, n_hi], redrawn while n > M/2 so that distinct keys
    exist at density at most 1/2.
    """
    u = unit(seed, 64 * count + 16)
    k = 0
    t = 0.0
    out = []
    for _ in range(count):
        t += -math.log(1.0 - u[k]) / rate_hz
        k += 1
        M = log_uniform_int(u[k], m_lo, m_hi)
        k += 1
        while True:
            n = log_uniform_int(u[k], n_lo, n_hi)
            k += 1
            if n <= M // 2:
                break
        out.append((t, n, M))
    return out
