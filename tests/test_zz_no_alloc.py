"""The allocation-free projection entry point, dialsort_reconstruct_noalloc.

Some callers of this library cannot allocate device memory when they call it
(a plugin handed only its input and output buffers by a framework that owns
all device memory, or a latency-critical loop that must not touch an
allocator).  For them the projection has a variant whose scratch sits in a
fixed library-owned device array.  This file checks, through the C ABI, that
it produces exactly what dialsort_reconstruct (caller workspace) produces, on
two calls in a row (the second reuses the array the first one left behind),
and that sizes beyond the fixed scratch are refused before anything runs.

It is collected last on purpose and must pass both alone in a fresh process
and after every other test.
"""
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


def _hist_on_device(ds, n, U, dist, stream_id):
    keys = gen.keys(n, U, dist, stream=stream_id)
    return ds.histogram(torch.from_numpy(keys.view(np.int32)).cuda(), U)


def _reference_projection(ds, H, U, n):
    """The existing entry point, with a caller-allocated workspace."""
    out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    ws = torch.empty(ds.reconstruct_workspace_size(U, n), dtype=torch.uint8, device="cuda")
    st = ds.lib().dialsort_reconstruct(H.data_ptr(), U, out.data_ptr(), n, ws.data_ptr(), ws.numel(),
                                       torch.cuda.current_stream().cuda_stream)
    assert st == ds.OK
    return out


def _noalloc_projection(ds, H, U, n):
    out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    st = ds.lib().dialsort_reconstruct_noalloc(H.data_ptr(), U, out.data_ptr(), n,
                                               torch.cuda.current_stream().cuda_stream)
    assert st == ds.OK
    return out


def test_noalloc_matches_workspace_entry_point_on_two_calls_in_a_row(ds):
    cases = [((1 << 20) + 11, 1 << 16, "zipf", 41), (300_007, 1 << 20, "uniform", 42)]
    for n, U, dist, sid in cases:  # two calls in a row; the second finds the first call's scratch contents
        H = _hist_on_device(ds, n, U, dist, sid)
        want = _reference_projection(ds, H, U, n)
        got = _noalloc_projection(ds, H, U, n)
        torch.cuda.synchronize()
        assert ds.stream_status() == ds.OK
        assert torch.equal(got, want)  # integer output: bit-exact, as every parity test here
    # and the same histogram twice, back to back
    H = _hist_on_device(ds, 123_457, 4099, "all_equal", 43)
    want = _reference_projection(ds, H, 4099, 123_457)
    a = _noalloc_projection(ds, H, 4099, 123_457)
    b = _noalloc_projection(ds, H, 4099, 123_457)
    torch.cuda.synchronize()
    assert torch.equal(a, want) and torch.equal(b, want)


def test_noalloc_matches_the_oracle_and_allocates_nothing(ds):
    n, U = (1 << 19) + 5, 1 << 14
    keys = gen.keys(n, U, "zipf", stream=44)
    H = ds.histogram(torch.from_numpy(keys.view(np.int32)).cuda(), U)
    first = _noalloc_projection(ds, H, U, n)  # the first call on a device looks up the scratch address
    torch.cuda.synchronize()
    # the direct check: the CPU oracle's projection of the same histogram, element by element
    want = oracle.reconstruct(H.cpu().numpy().view(np.uint32), U)
    assert np.array_equal(first.cpu().numpy().view(np.uint32), want)
    # the property the entry point exists for: a further call takes no device memory
    out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    st = ds.lib().dialsort_reconstruct_noalloc(H.data_ptr(), U, out.data_ptr(), n,
                                               torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    assert st == ds.OK and free_after == free_before
    assert np.array_equal(out.cpu().numpy().view(np.uint32), want)


def test_noalloc_classifies_h_and_out_like_the_workspace_entry_point(ds):
    """A histogram in plain (pageable) host memory: refused where the GPU cannot read host page
    tables, read across the CPU-GPU link where it can -- exactly as dialsort_reconstruct does."""
    n, U = 4099, 256
    keys = gen.keys(n, U, "uniform", stream=45)
    buf = np.zeros(U + 4, np.uint32)  # a 16-byte aligned view into plain host memory
    off = (-buf.ctypes.data % 16) // 4
    H_host = buf[off:off + U]
    H_host[:] = oracle.histogram(keys, U)[0]
    out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    L = ds.lib()
    st = L.dialsort_reconstruct_noalloc(H_host.ctypes.data, U, out.data_ptr(), n, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    ws = torch.empty(ds.reconstruct_workspace_size(U, n), dtype=torch.uint8, device="cuda")
    out2 = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    st2 = L.dialsort_reconstruct(H_host.ctypes.data, U, out2.data_ptr(), n, ws.data_ptr(), ws.numel(),
                                 torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert st == st2
    if L.dialsort_pageable_host_access() == 1:
        assert st == ds.OK
        assert np.array_equal(out.cpu().numpy().view(np.uint32), oracle.reconstruct(H_host, U))
    else:
        assert st == ds.ERR_INVALID_ARG


def test_noalloc_refuses_sizes_beyond_its_scratch(ds):
    L = ds.lib()
    H = torch.zeros(16, dtype=torch.int32, device="cuda")
    out = torch.zeros(16, dtype=torch.int32, device="cuda")
    U, n = 1 << 27, (1 << 31)
    assert L.dialsort_reconstruct_workspace_size(U, n) > (2 << 20)
    # checked on the host before any launch: H and out are never touched
    st = L.dialsort_reconstruct_noalloc(H.data_ptr(), U, out.data_ptr(), n, torch.cuda.current_stream().cuda_stream)
    assert st == ds.ERR_WORKSPACE
