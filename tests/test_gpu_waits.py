"""Bounded device waits: a look-back whose predecessor never publishes gives up after its spin
limit, records DIALSORT_ERR_TIMEOUT in the error word and returns; the context stays usable."""
import time

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


@pytest.mark.parametrize("which", [0, 1], ids=["offset-scan", "radix-pass"])
def test_wait_runs_out_reports_timeout_and_context_survives(ds, which):
    L = ds.lib()
    ws = torch.empty(L.dialsort_selftest_workspace_size(), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    assert ds.stream_status() == ds.OK  # start from a clear error word
    t0 = time.perf_counter()
    assert L.dialsort_selftest_wait_timeout(which, ws.data_ptr(), ws.numel(), stream.cuda_stream) == ds.OK
    assert ds.stream_status() == ds.ERR_TIMEOUT  # synchronises, reads and clears
    assert time.perf_counter() - t0 < 30.0
    assert ds.stream_status() == ds.OK  # cleared by the read
    keys = gen.keys(1_000_003, 5000, "zipf", stream=9500 + which)  # the context still sorts correctly
    out = ds.sort(torch.from_numpy(keys.view(np.int32)).cuda(), 5000)
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), oracle.sort(keys, 5000))
    assert ds.stream_status() == ds.OK


def test_selftest_rejects_bad_arguments(ds):
    L = ds.lib()
    assert L.dialsort_selftest_wait_timeout(2, None, 0, None) == ds.ERR_INVALID_ARG
    assert L.dialsort_selftest_wait_timeout(0, None, 0, None) == ds.ERR_WORKSPACE
