"""Keys read from, and output written to, host memory by the kernels themselves (no staging copy):
results equal the oracle bit for bit, for every ingestion regime and both key widths."""
import ctypes

import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ds():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    import paper_2605_16667_gb300 as ds

    return ds


def pinned(a):
    view = a.view(np.int32) if a.dtype == np.uint32 else a.view(np.int16)
    t = torch.empty(a.size, dtype=torch.int32 if a.dtype == np.uint32 else torch.int16, pin_memory=True)
    t.copy_(torch.from_numpy(view))
    return t


def as_np(t, dtype):
    return t.cpu().numpy().view(dtype)


@pytest.mark.parametrize("n,U,dist", [
    (100_003, 200, "zipf"),                # shared-memory regime, short input
    ((1 << 22) + 5, 4096, "uniform"),      # shared-memory regime, ragged tail
    ((1 << 21) + 3, 1 << 16, "zipf"),      # 16-bit packed sub-histograms
    ((1 << 22) + 1, 1 << 20, "uniform"),   # two-level regime (keys read once by the partition pass)
    ((1 << 21) + 9, 3 << 20, "all_equal"),
    (5_000, 1 << 22, "uniform"),           # L2 regime (n too small for two-level)
])
def test_sort_host_keys_host_out(ds, n, U, dist):
    keys = gen.keys(n, U, dist, stream=7100 + n % 97)
    hk = pinned(keys)
    out = ds.sort(hk, U)  # out allocated pinned as well
    assert not out.is_cuda and out.is_pinned()
    torch.cuda.synchronize()
    assert ds.stream_status() == ds.OK
    np.testing.assert_array_equal(as_np(out, np.uint32), oracle.sort(keys, U))


def test_sort_host_in_place_and_u16(ds):
    keys = gen.keys((1 << 20) + 77, 1 << 16, "zipf", width=2, stream=7201)
    hk = pinned(keys)
    ds.sort(hk, 1 << 16, out=hk)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(as_np(hk, np.uint16), oracle.sort(keys, 1 << 16))


def test_mixed_host_and_device(ds):
    U = 70_000
    keys = gen.keys(3_000_001, U, "uniform", stream=7202)
    H = ds.histogram(pinned(keys), U)  # host keys, device H
    assert H.is_cuda
    H_ref, _ = oracle.histogram(keys, U)
    np.testing.assert_array_equal(as_np(H, np.uint32), H_ref)
    hout = torch.empty(keys.size, dtype=torch.int32, pin_memory=True)
    ds.reconstruct(H, U, keys.size, out=hout)  # device H, host output
    dkeys = torch.from_numpy(keys.view(np.int32)).cuda()
    dout = ds.sort(dkeys, U, out=torch.empty(keys.size, dtype=torch.int32, pin_memory=True))  # device keys, host out
    torch.cuda.synchronize()
    ref = oracle.reconstruct(H_ref, U)
    np.testing.assert_array_equal(as_np(hout, np.uint32), ref)
    np.testing.assert_array_equal(as_np(dout, np.uint32), ref)


def test_out_of_range_key_in_host_memory(ds):
    keys = gen.keys(1 << 20, 1000, "uniform", stream=7203)
    keys[4242] = 1000
    H = ds.histogram(pinned(keys), 1000)
    assert ds.stream_status() == ds.ERR_KEY_RANGE
    np.testing.assert_array_equal(as_np(H, np.uint32), oracle.histogram(keys, 1000)[0])


def test_pageable_host_memory_follows_the_device_attribute(ds):
    """Plain (pageable) host memory: sorted by the kernels where the device reads host page tables,
    refused on the host (INVALID_ARG, nothing launched) where it does not."""
    U, n = 5000, (1 << 20) + 3
    keys = gen.keys(n, U, "zipf", stream=7204)
    out = np.zeros(n, dtype=np.uint32)
    ws = torch.empty(ds.sort_workspace_size(n, U), dtype=torch.uint8, device="cuda")
    st = ds.lib().dialsort_sort(keys.ctypes.data, n, U, out.ctypes.data, ws.data_ptr(), ws.numel(),
                                torch.cuda.current_stream().cuda_stream)
    if not ds.pageable_host_access():
        assert st == ds.ERR_INVALID_ARG
        return
    assert st == ds.OK
    torch.cuda.synchronize()
    assert ds.stream_status() == ds.OK
    np.testing.assert_array_equal(out, oracle.sort(keys, U))
