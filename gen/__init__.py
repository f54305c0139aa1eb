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
