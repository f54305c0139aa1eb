"""DialSort CPU oracle -- TEST INFRASTRUCTURE ONLY.

Plain, slow, single-threaded definitions of what the DialSort hot path
computes, written in C (``dialsort_oracle.c``) from the paper's equations and
wrapped here with ctypes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the CUDA product path
never does, and the two share no code.

Functions and the passages they follow:

* ``histogram``   -- Eq. (1), ingestion, with H zeroed first (Theorem
  "Sequential complexity": the Theta(U) initialisation).
* ``reconstruct`` -- Eq. (2), ordered projection.
* ``sort``        -- Eq. (1) then Eq. (2) (Theorem "Correctness of DialSort").
* ``offsets``     -- the cursor of the sequential projection of Eq. (2) on
  reaching each k: O[k] = sum_{j<k} H[j].
* ``crn_level`` / ``crn`` -- Definition "CRN level transition" with the node
  rule of Eqs. (3)-(4).
* ``accumulate``  -- Eq. (1) without the zeroing (a stream of batches ingested
  into one H).
* ``sort_mapped`` -- Prop. "General Self-Indexing Principle": Eq. (1) on
  phi(key), then Eq. (2) emitting phi_inv(i).
* ``radix_sort``  -- DialSort-Radix of Sec. "Full int32 range": four stable
  counting passes (Eq. (1) on a base-256 digit, then placement at the digit's
  cursor), least significant digit first; int32 keys sort as signed.
* ``frequency`` / ``presence`` / ``range_count`` -- the queries of Sec.
  "Canonical ordered state", answered from H alone (range bounds inclusive).

Every function is pinned by ``tests/test_oracle_pins.py`` against the paper's
worked examples, brute force, library routines and the theorems' invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dialsort_oracle.c")
_LIB = os.path.join(_HERE, "libdialsort_oracle.so")
_lib = None

_P = ctypes.c_void_p
_U64 = ctypes.c_uint64
_U32 = ctypes.c_uint32
_SZ = ctypes.c_size_t


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (single-threaded, no vectorisation flags)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        for name in ("oracle_histogram_u32", "oracle_histogram_u16"):
            f = getattr(lib, name)
            f.restype = _U64
            f.argtypes = [_P, _U64, _U32, _P]
        for name in ("oracle_reconstruct_u32", "oracle_reconstruct_u16"):
            f = getattr(lib, name)
            f.restype = _U64
            f.argtypes = [_P, _U32, _P, _U64]
        lib.oracle_offsets.restype = None
        lib.oracle_offsets.argtypes = [_P, _U32, _P]
        lib.oracle_crn_level.restype = _SZ
        lib.oracle_crn_level.argtypes = [_P, _P, _SZ, _P, _P]
        lib.oracle_crn.restype = _SZ
        lib.oracle_crn.argtypes = [_P, _P, _SZ, _P, _P]
        for name in ("oracle_accumulate_u32", "oracle_accumulate_u16"):
            f = getattr(lib, name)
            f.restype = _U64
            f.argtypes = [_P, _U64, _U32, _P]
        for name in ("oracle_frequency", "oracle_presence"):
            f = getattr(lib, name)
            f.restype = None
            f.argtypes = [_P, _U32, _P, _U64, _P]
        lib.oracle_sort_mapped.restype = _U64
        lib.oracle_sort_mapped.argtypes = [_P, _U64, _P, _U32, _P, _U32, _P, _P]
        lib.oracle_radix_sort.restype = None
        lib.oracle_radix_sort.argtypes = [_P, _U64, ctypes.c_int, _P, _P]
        lib.oracle_range_count.restype = None
        lib.oracle_range_count.argtypes = [_P, _U32, _P, _P, _U64, _P]
        _lib = lib
    return _lib


def _c(a: np.ndarray, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def histogram(keys: np.ndarray, U: int) -> tuple[np.ndarray, int]:
    """Eq. (1). Returns (H as uint32[U], number of keys >= U that were skipped)."""
    keys = np.asarray(keys)
    H = np.empty(U, dtype=np.uint32)
    if keys.dtype == np.uint16:
        k = _c(keys, np.uint16)
        skipped = _load().oracle_histogram_u16(k.ctypes.data, k.size, U, H.ctypes.data)
    else:
        k = _c(keys, np.uint32)
        skipped = _load().oracle_histogram_u32(k.ctypes.data, k.size, U, H.ctypes.data)
    return H, int(skipped)


def reconstruct(H: np.ndarray, U: int | None = None, width: int = 4, cap: int | None = None) -> np.ndarray:
    """Eq. (2). Emits k exactly H[k] times for k = 0..U-1 (uint32 or uint16 output)."""
    H = _c(H, np.uint32)
    U = H.size if U is None else U
    total = int(H[:U].astype(np.uint64).sum())
    cap = total if cap is None else cap
    if width == 4:
        out = np.empty(cap, dtype=np.uint32)
        n = _load().oracle_reconstruct_u32(H.ctypes.data, U, out.ctypes.data, cap)
    else:
        out = np.empty(cap, dtype=np.uint16)
        n = _load().oracle_reconstruct_u16(H.ctypes.data, U, out.ctypes.data, cap)
    assert n == total
    return out


def sort(keys: np.ndarray, U: int) -> np.ndarray:
    """Eq. (1) followed by Eq. (2)."""
    keys = np.asarray(keys)
    H, _ = histogram(keys, U)
    return reconstruct(H, U, width=2 if keys.dtype == np.uint16 else 4)


def accumulate(keys: np.ndarray, U: int, H: np.ndarray) -> tuple[np.ndarray, int]:
    """Eq. (1) without zeroing: returns (H + counts of keys, keys >= U skipped); H is not modified."""
    keys = np.asarray(keys)
    H = _c(H, np.uint32).copy()
    assert H.size == U
    if keys.dtype == np.uint16:
        k = _c(keys, np.uint16)
        skipped = _load().oracle_accumulate_u16(k.ctypes.data, k.size, U, H.ctypes.data)
    else:
        k = _c(keys, np.uint32)
        skipped = _load().oracle_accumulate_u32(k.ctypes.data, k.size, U, H.ctypes.data)
    return H, int(skipped)


def sort_mapped(keys: np.ndarray, U: int, phi=None, phi_inv=None) -> tuple[np.ndarray, np.ndarray, int]:
    """Prop. "General Self-Indexing Principle": count each key at phi(key), emit phi_inv(i) H[i] times.

    phi: array of M indices (0xffffffff = not in the domain) or None (identity); phi_inv: U values or
    None (identity).  Returns (out in the keys' dtype, H, number of keys not counted)."""
    keys = np.asarray(keys)
    k = np.ascontiguousarray(keys, dtype=np.uint32)
    H = np.empty(U, dtype=np.uint32)
    out = np.empty(k.size, dtype=np.uint32)
    ph = None if phi is None else np.ascontiguousarray(phi, dtype=np.uint32)
    inv = None if phi_inv is None else np.ascontiguousarray(phi_inv, dtype=np.uint32)
    skipped = _load().oracle_sort_mapped(k.ctypes.data, k.size, None if ph is None else ph.ctypes.data,
                                         0 if ph is None else ph.size, None if inv is None else inv.ctypes.data,
                                         U, out.ctypes.data, H.ctypes.data)
    total = k.size - int(skipped)
    return out[:total].astype(keys.dtype), H, int(skipped)


def radix_sort(keys: np.ndarray) -> np.ndarray:
    """DialSort-Radix: LSD base 256, four stable counting passes; int32 keys sort as signed."""
    keys = np.asarray(keys)
    assert keys.dtype in (np.int32, np.uint32)
    k = np.ascontiguousarray(keys).view(np.uint32)
    out = np.empty(k.size, dtype=np.uint32)
    tmp = np.empty(k.size, dtype=np.uint32)
    _load().oracle_radix_sort(k.ctypes.data, k.size, 1 if keys.dtype == np.int32 else 0, out.ctypes.data,
                              tmp.ctypes.data)
    return out.view(keys.dtype)


def frequency(H: np.ndarray, q) -> np.ndarray:
    """frequency(k) = H[k] for each query key (0 outside [0, U))."""
    H = _c(H, np.uint32)
    q = _c(q, np.uint32)
    out = np.empty(q.size, dtype=np.uint32)
    _load().oracle_frequency(H.ctypes.data, H.size, q.ctypes.data, q.size, out.ctypes.data)
    return out


def presence(H: np.ndarray, q) -> np.ndarray:
    """presence(k) = 1 if H[k] > 0 else 0, as uint8."""
    H = _c(H, np.uint32)
    q = _c(q, np.uint32)
    out = np.empty(q.size, dtype=np.uint8)
    _load().oracle_presence(H.ctypes.data, H.size, q.ctypes.data, q.size, out.ctypes.data)
    return out


def range_count(H: np.ndarray, a, b) -> np.ndarray:
    """range-count(a, b) = sum of H[k] for a <= k <= b (inclusive), as uint64."""
    H = _c(H, np.uint32)
    a = _c(a, np.uint32)
    b = _c(b, np.uint32)
    assert a.size == b.size
    out = np.empty(a.size, dtype=np.uint64)
    _load().oracle_range_count(H.ctypes.data, H.size, a.ctypes.data, b.ctypes.data, a.size, out.ctypes.data)
    return out


def offsets(H: np.ndarray, U: int | None = None) -> np.ndarray:
    """O[k] = sum_{j<k} H[j] for k = 0..U, as uint64[U+1]."""
    H = _c(H, np.uint32)
    U = H.size if U is None else U
    O = np.empty(U + 1, dtype=np.uint64)
    _load().oracle_offsets(H.ctypes.data, U, O.ctypes.data)
    return O


def crn_level(keys, counts) -> tuple[np.ndarray, np.ndarray]:
    """One level of Definition "CRN level transition"."""
    k = _c(keys, np.uint32)
    c = _c(counts, np.uint64)
    ko = np.empty(max(k.size, 1), dtype=np.uint32)
    co = np.empty(max(k.size, 1), dtype=np.uint64)
    m = _load().oracle_crn_level(k.ctypes.data, c.ctypes.data, k.size, ko.ctypes.data, co.ctypes.data)
    return ko[:m].copy(), co[:m].copy()


def crn(keys, counts=None) -> tuple[np.ndarray, np.ndarray]:
    """ceil(log2 k) CRN levels over k lanes; returns the surviving (key, count) items."""
    k = _c(keys, np.uint32).copy()
    c = np.ones(k.size, dtype=np.uint64) if counts is None else _c(counts, np.uint64).copy()
    sk = np.empty(max(k.size, 1), dtype=np.uint32)
    sc = np.empty(max(k.size, 1), dtype=np.uint64)
    m = _load().oracle_crn(k.ctypes.data, c.ctypes.data, k.size, sk.ctypes.data, sc.ctypes.data)
    return k[:m].copy(), c[:m].copy()
