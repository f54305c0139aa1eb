"""ctypes binding of libdialsort.so: the C ABI of include/dialsort.h, same names.

Argument marshalling only.  Every step of the DialSort path runs in the
library's CUDA kernels; there is no CPU fallback.  Loading fails loudly when
the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdialsort.so")

P = ctypes.c_void_p
U64 = ctypes.c_uint64
U32 = ctypes.c_uint32
SZ = ctypes.c_size_t
INT = ctypes.c_int
STATUS = ctypes.c_int


class dialsort_hist_config_t(ctypes.Structure):
    _fields_ = [("regime", U32), ("crn", U32), ("blocks", U32), ("threads", U32), ("replicas", U32),
                ("cluster", U32), ("skew", U32)]


class dialsort_skew_t(ctypes.Structure):
    _fields_ = [("samples", U32), ("equal_neighbours", U32), ("neighbour_pairs", U32), ("top_multiplicity", U32),
                ("skew_class", U32), ("reserved", U32)]


class dialsort_instance_t(ctypes.Structure):
    _fields_ = [("keys", P), ("H", P), ("out", P), ("n", U64), ("U", U32), ("key_bytes", U32), ("skew", U32),
                ("regime", U32)]


class dialsort_server_cfg_t(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", U64), ("max_slots", U32), ("reserved", U32), ("idle_timeout_ns", U64)]


class dialsort_request_t(ctypes.Structure):
    _fields_ = [("keys", P), ("n", U64), ("U", U32), ("key_bytes", U32), ("kind", U32), ("skew", U32)]


class dialsort_result_t(ctypes.Structure):
    _fields_ = [("H", P), ("out", P), ("submit_ns", U64), ("admit_ns", U64), ("done_ns", U64), ("status", U32),
                ("reserved", U32)]


class dialsort_trace_entry_t(ctypes.Structure):
    _fields_ = [("keys", P), ("n", U64), ("U", U32), ("key_bytes", U32), ("kind", U32), ("reserved", U32),
                ("arrival_ns", U64)]


class dialsort_trace_result_t(ctypes.Structure):
    _fields_ = [("arrival_ns", U64), ("done_ns", U64), ("status", U32), ("reserved", U32)]


# name -> (restype, argtypes); mirrors include/dialsort.h
SIGNATURES = {
    "dialsort_histogram": (STATUS, [P, U64, U32, P, P]),
    "dialsort_histogram_u16": (STATUS, [P, U64, U32, P, P]),
    "dialsort_histogram_ex": (STATUS, [P, U32, U64, U32, P, P, P]),
    "dialsort_plan_histogram": (STATUS, [U64, U32, U32, U32, P]),
    "dialsort_probe_skew": (STATUS, [P, U32, U64, U32, P, P]),
    "dialsort_probe_skew_batched": (STATUS, [P, U32, P]),
    "dialsort_tune_table_load": (STATUS, [ctypes.c_char_p]),
    "dialsort_tune_table_size": (U32, []),
    "dialsort_histogram_workspace_size": (SZ, [U64, U32, U32]),
    "dialsort_histogram_ws": (STATUS, [P, U32, U64, U32, P, P, P, SZ, P]),
    "dialsort_reconstruct_workspace_size": (SZ, [U32, U64]),
    "dialsort_reconstruct": (STATUS, [P, U32, P, U64, P, SZ, P]),
    "dialsort_reconstruct_u16": (STATUS, [P, U32, P, U64, P, SZ, P]),
    "dialsort_offsets": (STATUS, [P, U32, U64, P, SZ, P]),
    "dialsort_read_chunk_offsets": (STATUS, [P, U32, U64, P, P]),
    "dialsort_reconstruct_noalloc": (STATUS, [P, U32, P, U64, P]),
    "dialsort_histogram_accumulate": (STATUS, [P, U32, U64, U32, P, P, SZ, P]),
    "dialsort_chunked_workspace_size": (SZ, [U64, U32, U32, U64, INT]),
    "dialsort_histogram_chunked": (STATUS, [P, U32, U64, U32, U64, P, P, SZ, P, P]),
    "dialsort_sort_chunked": (STATUS, [P, U32, U64, U32, U64, P, P, SZ, P, P]),
    "dialsort_sort_mapped_workspace_size": (SZ, [U64, U32]),
    "dialsort_sort_mapped": (STATUS, [P, U32, U64, P, U32, P, U32, P, P, SZ, P]),
    "dialsort_radix_workspace_size": (SZ, [U64]),
    "dialsort_radix_sort_i32": (STATUS, [P, U64, P, P, SZ, P]),
    "dialsort_radix_sort_u32": (STATUS, [P, U64, P, P, SZ, P]),
    "dialsort_frequency": (STATUS, [P, U32, P, U64, P, P]),
    "dialsort_presence": (STATUS, [P, U32, P, U64, P, P]),
    "dialsort_range_count": (STATUS, [P, U32, P, P, U64, P, P]),
    "dialsort_sort_workspace_size": (SZ, [U64, U32]),
    "dialsort_sort": (STATUS, [P, U64, U32, P, P, SZ, P]),
    "dialsort_sort_u16": (STATUS, [P, U64, U32, P, P, SZ, P]),
    "dialsort_sort_ex": (STATUS, [P, U32, U64, U32, P, P, P, SZ, P]),
    "dialsort_sort_stage_times": (STATUS, [P, U32, U64, U32, P, P, SZ, P, P, P]),
    "dialsort_sort_histogram": (P, [P]),
    "dialsort_batch_create": (STATUS, [P, U32, INT, P]),
    "dialsort_batch_workspace_size": (SZ, [P]),
    "dialsort_batch_launch": (STATUS, [P, P, SZ, P]),
    "dialsort_batch_destroy": (STATUS, [P]),
    "dialsort_batch_describe": (STATUS, [P, U32, P, P]),
    "dialsort_batched_workspace_size": (SZ, [P, U32, INT]),
    "dialsort_batched": (STATUS, [P, U32, INT, P, SZ, P]),
    "dialsort_histogram_batched": (STATUS, [P, U32, P, SZ, P]),
    "dialsort_sort_batched": (STATUS, [P, U32, P, SZ, P]),
    "dialsort_server_create": (STATUS, [P, P]),
    "dialsort_server_submit": (STATUS, [P, P, P]),
    "dialsort_server_poll": (STATUS, [P, U64, P]),
    "dialsort_server_wait": (STATUS, [P, U64, U64, P]),
    "dialsort_server_release": (STATUS, [P, U64]),
    "dialsort_server_destroy": (STATUS, [P]),
    "dialsort_replay": (STATUS, [P, U32, INT, P, P, P]),
    "dialsort_stream_status": (STATUS, [P, INT]),
    "dialsort_status_string": (ctypes.c_char_p, [STATUS]),
    "dialsort_device_sm_count": (INT, []),
    "dialsort_pageable_host_access": (INT, []),
    "dialsort_selftest_workspace_size": (SZ, []),
    "dialsort_selftest_wait_timeout": (STATUS, [INT, P, SZ, P]),
    "dialsort_version": (ctypes.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libdialsort.so and attach the signatures; raises if it is missing."""
    global _lib
    if _lib is not None and path == LIB_PATH:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built: run `python -c 'import __graft_entry__ as g; g.build()'` first "
                           "(DialSort has no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path == LIB_PATH:
        _lib = lib
    return lib


def __getattr__(name):
    # native.dialsort_histogram(...) etc. resolve to the C functions
    if name.startswith("dialsort_"):
        return getattr(load(), name)
    raise AttributeError(name)
