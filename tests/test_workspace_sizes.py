"""Host-side size queries of the C ABI at extreme sizes (no GPU): every workspace is a whole number of
256-byte blocks, holds what its layout must (H, one 16-bit low part per key in the two-level path, the
radix ping-pong keys), and does not wrap around at the largest n and U the API accepts."""
from __future__ import annotations

import os

import pytest

NS = [0, 1, 8191, 8192, 8193, 1 << 20, (1 << 20) + 7, 1 << 28, (1 << 31) + 5, (1 << 32) - 1]
US = [1, 2, 255, 256, 1024, 4096, 65536, 65537, 1 << 20, (1 << 20) + 1, 1 << 24, 1 << 26, 1 << 31, (1 << 32) - 1]


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g

    g.build()
    import paper_2605_16667_gb300 as ds

    return ds.lib()


@pytest.mark.parametrize("U", US)
def test_sort_and_reconstruct_workspaces(lib, U):
    for n in NS:
        s = lib.dialsort_sort_workspace_size(n, U)
        r = lib.dialsort_reconstruct_workspace_size(U, n)
        h = lib.dialsort_histogram_workspace_size(n, U, 4)
        assert s % 256 == 0 and r % 256 == 0
        assert s >= 4 * U  # H lives at the start of the sort workspace
        assert s >= r  # the sort runs the projection in its own workspace
        chunks = -(-U // 1024)
        assert r >= 8 * (chunks + 1)  # one 64-bit run start per 1024-bin chunk, plus the total
        for size in (s, r, h):
            assert size < 1 << 48  # no wrap-around into a huge size_t


def test_two_level_workspace_holds_the_low_parts(lib):
    import paper_2605_16667_gb300 as ds

    ds.tune_table_load(None)  # the cost model's choice (a measured table may prefer the L2 regime)
    try:
        for n, U in [(1 << 20, 1 << 20), (1 << 28, 1 << 20), (1 << 27, 1 << 24), ((1 << 32) - 1, 1 << 26)]:
            assert ds.plan_histogram(n, U)["regime_name"] == "two_level"
            h = lib.dialsort_histogram_workspace_size(n, U, 4)
            tiles = -(-n // 8192)
            assert h >= 2 * 8192 * tiles  # 16-bit low parts, tile-major
    finally:
        ds.tune_table_load(ds.TUNE_TABLE if os.path.exists(ds.TUNE_TABLE) else None)


def test_radix_workspace_holds_the_ping_pong_keys(lib):
    for n in NS:
        w = lib.dialsort_radix_workspace_size(n)
        assert w % 256 == 0 and w >= 4 * n and w < 1 << 48
