"""Chunked ingestion from host memory, overlapped with the copies (dialsort_histogram_chunked /
dialsort_sort_chunked), against the CPU oracle element by element: H += histogram of the keys
(oracle.accumulate) and the sorted output (oracle.reconstruct of the oracle's histogram)."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def ds():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    import paper_2605_16667_gb300 as ds

    assert ds.stream_status() == ds.OK
    return ds


def host_tensor(a: np.ndarray, pinned: bool):
    t = torch.from_numpy(a.view(np.int32) if a.dtype == np.uint32 else a.view(np.int16))
    return t.pin_memory() if pinned else t.clone()


CASES = [
    (0, 256, 1 << 20), (1, 256, 1 << 20), ((1 << 20) - 1, 1 << 12, 1 << 20), (1 << 20, 1 << 12, 1 << 20),
    ((1 << 20) + 1, 1 << 16, 1 << 20), (5 * (1 << 20) + 12345, 1 << 20, 1 << 20),
    (3 * (1 << 21) + 7, 3 * (1 << 20) - 1, (1 << 21) + 3), (4 * (1 << 20) + 99, 1 << 24, 1 << 20),
    (2_000_001, 1000, 65536 + 5),
]


@pytest.mark.parametrize("n,U,chunk", CASES)
@pytest.mark.parametrize("dist", ["uniform", "zipf", "sorted"])
def test_histogram_chunked_matches_oracle_accumulate(ds, n, U, chunk, dist):
    keys = gen.keys(n, U, dist, stream=71)
    H0 = gen.keys(U, 1000, "uniform", stream=72)  # counts already in H
    H = torch.from_numpy(H0.view(np.int32).copy()).cuda()
    s, cs = torch.cuda.Stream(), torch.cuda.Stream()
    with torch.cuda.stream(s):
        ds.histogram_chunked(host_tensor(keys, True), U, H, chunk_keys=chunk, stream=s, copy_stream=cs)
    s.synchronize()
    assert ds.stream_status() == ds.OK
    want, skipped = oracle.accumulate(keys, U, H0.copy())
    assert skipped == 0
    np.testing.assert_array_equal(H.cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("n,U,chunk", [(3 * (1 << 20) + 5, 1 << 16, 1 << 20), (777_777, 300, 100_000)])
@pytest.mark.parametrize("pinned", [True, False])
def test_histogram_chunked_u16_and_pageable(ds, n, U, chunk, pinned):
    keys = gen.keys(n, U, "zipf", width=2, stream=73)
    H = torch.zeros(U, dtype=torch.int32, device="cuda")
    s, cs = torch.cuda.Stream(), torch.cuda.Stream()
    ds.histogram_chunked(host_tensor(keys, pinned), U, H, chunk_keys=chunk, stream=s, copy_stream=cs)
    s.synchronize()
    want, _ = oracle.accumulate(keys, U, np.zeros(U, dtype=np.uint32))
    np.testing.assert_array_equal(H.cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("n,U,chunk,width", [
    (0, 10, 1 << 20, 4), (4 * (1 << 20) + 3, 1 << 20, 1 << 20, 4), ((1 << 22) + 1, 1 << 12, 3 * (1 << 19), 4),
    (3_000_017, 65536, 1 << 20, 2), (1_000_003, 1 << 24, 250_000, 4),
])
@pytest.mark.parametrize("out_on", ["device", "pinned"])
def test_sort_chunked_matches_oracle(ds, n, U, chunk, width, out_on):
    keys = gen.keys(n, U, "zipf" if width == 2 else "uniform", width=width, stream=74)
    dt = torch.int32 if width == 4 else torch.int16
    out = torch.empty(n, dtype=dt, device="cuda") if out_on == "device" else torch.empty(n, dtype=dt, pin_memory=True)
    s, cs = torch.cuda.Stream(), torch.cuda.Stream()
    ds.sort_chunked(host_tensor(keys, True), U, out, chunk_keys=chunk, stream=s, copy_stream=cs)
    s.synchronize()
    assert ds.stream_status() == ds.OK
    H_ref, _ = oracle.histogram(keys, U)
    want = oracle.reconstruct(H_ref, U, width)
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32 if width == 4 else np.uint16), want)


def test_chunked_argument_errors(ds):
    keys = torch.zeros(1000, dtype=torch.int32).pin_memory()
    H = torch.zeros(16, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    with pytest.raises(ds.DialSortError):  # the copy stream must differ from the ingesting stream
        ds.histogram_chunked(keys, 16, H, chunk_keys=100, stream=s, copy_stream=s)
    with pytest.raises(ds.DialSortError):  # chunk of 0 keys
        ds.histogram_chunked(keys, 16, H, chunk_keys=0, stream=s, copy_stream=torch.cuda.Stream())
    with pytest.raises(TypeError):  # device keys: use histogram / histogram_accumulate
        ds.histogram_chunked(keys.cuda(), 16, H)
