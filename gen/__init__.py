"""Seeded synthetic key generators (shared input module).

Both the CPU oracle tests and the GPU path draw their inputs from here, so the
two sides see the same keys.  The module only draws random keys and sizes; it
holds none of the sorting method's arithmetic.  The C source next to this file
is compiled on first use with the host compiler (``build()``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dialsort_gen.c")
_LIB = os.path.join(_HERE, "libdialsort_gen.so")

UNIFORM, ZIPF, ALL_EQUAL, SORTED, REVERSE, RUNS, PAPER_SKEW, ZIPF_PERM = range(8)
DISTS = {
    "uniform": UNIFORM,
    "zipf": ZIPF,
    "all_equal": ALL_EQUAL,
    "sorted": SORTED,
    "reverse": REVERSE,
    "runs": RUNS,
    "paper_skew": PAPER_SKEW,
    "zipf_perm": ZIPF_PERM,
}

#: base seed of the paper's benchmark protocol (Sec. "Methodology")
BASE_SEED = 20260321

_lib = None


def build(force: bool = False) -> str:
    """Compile the generator library with gcc (quick; no GPU needed)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.gen_keys.restype = ctypes.c_int
        lib.gen_keys.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64]
        lib.gen_loguniform.restype = None
        lib.gen_loguniform.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_uint64, ctypes.c_uint64]
        lib.gen_unit.restype = None
        lib.gen_unit.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        lib.gen_u64.restype = None
        lib.gen_u64.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        _lib = lib
    return _lib


def keys(n: int, U: int, dist: str = "uniform", *, width: int = 4, param: float | None = None,
         seed: int = BASE_SEED, stream: int = 0, out: np.ndarray | None = None) -> np.ndarray:
    """Draw n keys in [0, U) as uint32 (width 4) or uint16 (width 2).

    ``param`` is the Zipf exponent (zipf, zipf_perm; default 1.2), the key for
    all_equal (default a fixed mid-universe value), or the block length for
    runs (default 2^20).
    """
    d = DISTS[dist]
    if param is None:
        if d in (ZIPF, ZIPF_PERM):
            param = 1.2
        elif d == ALL_EQUAL:
            param = float(0x5A5A5 % U)
        else:
            param = 0.0
    dtype = np.uint32 if width == 4 else np.uint16
    if out is None:
        out = np.empty(n, dtype=dtype)
    assert out.dtype == dtype and out.size >= n and out.flags.c_contiguous
    if n:
        rc = _load().gen_keys(out.ctypes.data, n, U, width, d, float(param), seed, stream)
        if rc != 0:
            raise ValueError(f"gen_keys failed ({rc}) for n={n} U={U} dist={dist} width={width}")
    return out[:n]


def loguniform(count: int, lo: float, hi: float, *, seed: int = BASE_SEED, stream: int = 0) -> np.ndarray:
    """floor(2^(lo + (hi-lo) u)) for u uniform in [0,1), clamped to [2^lo, 2^hi]."""
    out = np.empty(count, dtype=np.uint64)
    if count:
        _load().gen_loguniform(out.ctypes.data, count, lo, hi, seed, stream)
    return out


def unit(count: int, *, seed: int = BASE_SEED, stream: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1)."""
    out = np.empty(count, dtype=np.float64)
    if count:
        _load().gen_unit(out.ctypes.data, count, seed, stream)
    return out


def words(count: int, *, seed: int = BASE_SEED, stream: int = 0) -> np.ndarray:
    """Raw 64-bit random words."""
    out = np.empty(count, dtype=np.uint64)
    if count:
        _load().gen_u64(out.ctypes.data, count, seed, stream)
    return out


# ---------------------------------------------------------------- workload recipes
# The batched and served workloads, drawn here so that the benchmark and the tests see the same
# instances.  Sizes, universes and choices only: no sorting arithmetic.

def batch_workload(count: int = 4096):
    """The batched configuration: count instances, n_i log-uniform in [2^10, 2^22], U_i log-uniform in
    [2^8, 2^20], each instance's distribution drawn uniformly from {uniform, Zipf s=1.2, all equal},
    uint32 keys.  Returns (ns, us, dists); batch_keys(i, ...) draws instance i's keys."""
    ns = loguniform(count, 10, 22, stream=4 * 16).astype(np.int64)
    us = loguniform(count, 8, 20, stream=4 * 16 + 1).astype(np.int64)
    picks = words(count, stream=4 * 16 + 2)
    dists = [["uniform", "zipf", "all_equal"][int(p % 3)] for p in picks]
    return ns, us, dists


def batch_keys(i: int, n: int, U: int, dist: str, out: np.ndarray | None = None) -> np.ndarray:
    """Keys of instance i of batch_workload()."""
    return keys(int(n), int(U), dist, stream=4 * 16 * 1000 + i, out=out)


SERVED_POOL_KEYS = 1 << 26


def served_trace(rate: float = 2000.0, seconds: float = 10.0, warm: float = 1.0):
    """The served configuration's request trace: Poisson arrivals at `rate` req/s for warm + seconds,
    n log-uniform [2^12, 2^26], U log-uniform [2^8, 2^24], uint32/uint16 keys 50/50 (uint16 => U <=
    2^16), sort/histogram 50/50, uniform/Zipf 1.2 50/50.  A request's keys are a slice of a pool:
    for each (distribution, width) one base array of 2^26 keys over the largest universe (2^24 for
    uint32, 2^16 for uint16), shifted right so that the keys lie in [0, 2^c), c = floor(log2 U); the
    slice starts at offsets[i] (16-byte aligned).  Returns a dict of per-request arrays."""
    count = int(rate * (seconds + warm))
    gaps = -np.log1p(-unit(count, stream=5 * 16)) / rate
    arrivals = np.cumsum(gaps)
    ns = loguniform(count, 12, 26, stream=5 * 16 + 1).astype(np.int64)
    us = loguniform(count, 8, 24, stream=5 * 16 + 2).astype(np.int64)
    w = words(count, stream=5 * 16 + 3)
    width = np.where(w & 1, 2, 4)
    us = np.where(width == 2, np.minimum(us, 65536), us)
    kind = np.where((w >> 1) & 1, "sort", "histogram")
    dist = np.where((w >> 2) & 1, "zipf", "uniform")
    offs = words(count, stream=5 * 16 + 4)
    cls = np.floor(np.log2(us)).astype(np.int64)
    start = np.array([int(offs[i] % (SERVED_POOL_KEYS - ns[i] + 1)) for i in range(count)], dtype=np.int64)
    start -= start % 8
    return {"arrivals": arrivals, "n": ns, "U": us, "width": width, "kind": kind, "dist": dist,
            "cls": cls, "start": start, "warm": warm}


def served_pool(dist: str, width: int) -> np.ndarray:
    """The base key pool of served_trace() for one (distribution, width): 2^26 keys over [0, 2^24)
    (uint32) or [0, 2^16) (uint16)."""
    top = 24 if width == 4 else 16
    return keys(SERVED_POOL_KEYS, 1 << top, dist, width=width, param=1.2 if dist == "zipf" else None,
                stream=5 * 16 + 8)


def served_request_keys(pool: np.ndarray, width: int, c: int, start: int, n: int) -> np.ndarray:
    """Keys of one served request: the pool slice [start, start + n) shifted into [0, 2^c)."""
    top = 24 if width == 4 else 16
    return (pool[start:start + n] >> (top - c)).astype(pool.dtype)
