"""Multi-threaded CPU DialSort (count on private histograms, expand by bin ranges) for the benchmark's
host-core throughput line.  Not the oracle, and not on the GPU path: only ``bench.py`` uses it."""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dialsort_cpu.c")
_LIB = os.path.join(_HERE, "libdialsort_cpu.so")
_lib = None


def build(force: bool = False) -> str:
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC]
    if subprocess.run(cmd[:3] + ["-fopenmp"] + cmd[3:], capture_output=True).returncode != 0:
        subprocess.run(cmd, check=True)  # no OpenMP on this host: one thread
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.cpu_dialsort.restype = ctypes.c_int64
        lib.cpu_dialsort.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int]
        lib.cpu_dialsort_threads.restype = ctypes.c_int
        lib.cpu_dialsort_threads.argtypes = []
        _lib = lib
    return _lib


def threads() -> int:
    """Threads a call with threads=0 uses (1 when the host compiler has no OpenMP)."""
    return _load().cpu_dialsort_threads()


def sort(keys: np.ndarray, U: int, out: np.ndarray | None = None, threads: int = 0) -> np.ndarray:
    k = np.ascontiguousarray(keys, dtype=np.uint32)
    if out is None:
        out = np.empty(k.size, dtype=np.uint32)
    written = _load().cpu_dialsort(k.ctypes.data, k.size, U, out.ctypes.data, threads)
    if written < 0:
        raise MemoryError("cpu_dialsort: no memory for the per-thread histograms")
    return out[:written]
