"""Host-side argument checks of the newer entry points (no GPU): each bad call is refused with its
status before any device is touched.  Pointers are small fake addresses; nothing is dereferenced."""
from __future__ import annotations

import ctypes

import pytest

INVALID, WORKSPACE = 1, 8
K, H, OUT, WS = 4096, 8192, 12288, 16384  # 256-byte aligned fake device addresses


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g

    g.build()
    import paper_2605_16667_gb300 as ds

    return ds.lib()


CASES = {
    # Eq. (1) accumulated batch after batch
    "accumulate: null keys with n > 0": (lambda L: L.dialsort_histogram_accumulate(None, 4, 10, 16, H, None, 0, None),
                                          INVALID),
    "accumulate: key width 3": (lambda L: L.dialsort_histogram_accumulate(K, 3, 10, 16, H, None, 0, None), INVALID),
    # Eq. (2) pieces
    "offsets: null H": (lambda L: L.dialsort_offsets(None, 16, 10, WS, 1 << 20, None), INVALID),
    "reconstruct: U = 0": (lambda L: L.dialsort_reconstruct(H, 0, OUT, 10, WS, 1 << 20, None), INVALID),
    "reconstruct_noalloc: null H": (lambda L: L.dialsort_reconstruct_noalloc(None, 16, OUT, 10, None), INVALID),
    "sort: n = 2^32": (lambda L: L.dialsort_sort(K, 1 << 32, 16, OUT, WS, 1 << 20, None), INVALID),
    "sort_u16: U > 2^16": (lambda L: L.dialsort_sort_u16(K, 10, 65537, OUT, WS, 1 << 20, None), INVALID),
    # DialSort-Radix
    "radix i32: null keys": (lambda L: L.dialsort_radix_sort_i32(None, 10, OUT, WS, 1 << 20, None), INVALID),
    "radix u32: null out": (lambda L: L.dialsort_radix_sort_u32(K, 10, None, WS, 1 << 20, None), INVALID),
    "radix: no workspace": (lambda L: L.dialsort_radix_sort_i32(K, 10, OUT, None, 0, None), WORKSPACE),
    "radix: workspace too small": (lambda L: L.dialsort_radix_sort_u32(K, 1000, OUT, WS, 256, None), WORKSPACE),
    # queries on H
    "frequency: null H": (lambda L: L.dialsort_frequency(None, 16, K, 4, OUT, None), INVALID),
    "presence: null queries": (lambda L: L.dialsort_presence(H, 16, None, 4, OUT, None), INVALID),
    "range_count: null lower bounds": (lambda L: L.dialsort_range_count(H, 16, None, OUT, 4, WS, None), INVALID),
    # mapped domains
    "sort_mapped: key width 3": (lambda L: L.dialsort_sort_mapped(K, 3, 10, None, 0, None, 16, OUT, WS, 1 << 20, None),
                                 INVALID),
    "sort_mapped: U = 0": (lambda L: L.dialsort_sort_mapped(K, 4, 10, None, 0, None, 0, OUT, WS, 1 << 20, None),
                           INVALID),
    # batched and served forms
    "batched: null instances": (lambda L: L.dialsort_batched(None, 3, 1, None, 0, None), INVALID),
    "batch_create: null instances": (lambda L: L.dialsort_batch_create(None, 5, 1, ctypes.byref(ctypes.c_void_p())),
                                     INVALID),
    "server_create: null config": (lambda L: L.dialsort_server_create(None, ctypes.byref(ctypes.c_void_p())), INVALID),
    "server_submit: null server": (lambda L: L.dialsort_server_submit(None, None, ctypes.byref(ctypes.c_uint64())),
                                   INVALID),
    "server_poll: null server": (lambda L: L.dialsort_server_poll(None, 0, None), INVALID),
    "server_destroy: null server": (lambda L: L.dialsort_server_destroy(None), INVALID),
    # bounded-wait self-test
    "selftest: unknown wait": (lambda L: L.dialsort_selftest_wait_timeout(7, WS, 1 << 20, None), INVALID),
}


@pytest.mark.parametrize("name", list(CASES))
def test_bad_call_is_refused_on_the_host(lib, name):
    call, want = CASES[name]
    assert call(lib) == want
