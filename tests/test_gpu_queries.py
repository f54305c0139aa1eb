"""Queries answered from H on the device (frequency, presence, range-count) and accumulating
ingestion: bit-exact against the oracle."""
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


def dev32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def u32(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("U,dist", [(1, "uniform"), (6, "zipf"), (4099, "zipf"), (1 << 16, "uniform"),
                                    ((1 << 20) + 3, "all_equal"), ((1 << 22) + 1, "uniform")])
def test_point_queries(ds, U, dist):
    keys = gen.keys(1_000_003, U, dist, stream=9000 + U % 89)
    H_ref, _ = oracle.histogram(keys, U)
    H = dev32(H_ref)
    q = gen.keys(300_007, U + 64, "uniform", stream=9001)  # some queries fall outside [0, U)
    q[:3] = [0, U - 1, 0xFFFFFFFF]
    dq = dev32(q)
    np.testing.assert_array_equal(u32(ds.frequency(H, U, dq)), oracle.frequency(H_ref, q))
    np.testing.assert_array_equal(ds.presence(H, U, dq).cpu().numpy(), oracle.presence(H_ref, q))


@pytest.mark.parametrize("U,dist", [(1, "uniform"), (7, "uniform"), (4099, "zipf"), ((1 << 20) + 3, "sorted"),
                                    (1 << 22, "uniform")])
def test_range_count(ds, U, dist):
    keys = gen.keys(2_000_001, U, dist, stream=9100 + U % 83)
    H_ref, _ = oracle.histogram(keys, U)
    H = dev32(H_ref)
    m = 3000
    a = gen.keys(m, U + 8, "uniform", stream=9101)
    b = gen.keys(m, U + 8, "uniform", stream=9102)
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    a, b = lo.copy(), hi.copy()
    a[:8] = [0, 0, 5, U - 1, 3, 0, U, 2]  # full range, empty (a > b), point, tail, clipped, beyond, a = b
    b[:8] = [U - 1, 0xFFFFFFFF, 4, U - 1, U + 100, 0, U + 3, 2]
    a[8:16] = np.arange(8)  # ragged head and tail lengths 0..7 around the 4-bin vector loads
    b[8:16] = np.minimum(np.arange(8) + np.arange(8), U + 1)
    got = u32(ds.range_count(H, U, dev32(a), dev32(b)))
    np.testing.assert_array_equal(got, oracle.range_count(H_ref, a, b))


def test_queries_empty_and_host_arrays(ds):
    U = 1000
    keys = gen.keys(50_000, U, "zipf", stream=9200)
    H_ref, _ = oracle.histogram(keys, U)
    H = dev32(H_ref)
    e = torch.empty(0, dtype=torch.int32, device="cuda")
    assert ds.frequency(H, U, e).numel() == 0
    assert ds.range_count(H, U, e, e).numel() == 0
    q = np.arange(U, dtype=np.uint32)
    hq = torch.from_numpy(q.view(np.int32)).pin_memory()
    hout = torch.empty(U, dtype=torch.int32, pin_memory=True)
    ds.frequency(H, U, hq, out=hout)  # host queries and answers, device H
    torch.cuda.synchronize()
    np.testing.assert_array_equal(hout.numpy().view(np.uint32), H_ref)


@pytest.mark.parametrize("U,width", [(3000, 4), ((1 << 20) + 7, 4), (1 << 16, 2), (1 << 24, 4)])
def test_accumulate_batches_equals_one_histogram(ds, U, width):
    n = (1 << 22) + 11
    keys = gen.keys(n, U, "zipf" if U < (1 << 21) else "uniform", width=width, stream=9300 + U % 79)
    dk = torch.from_numpy(keys.view(np.int32 if width == 4 else np.int16)).cuda()
    H = torch.zeros(U, dtype=torch.int32, device="cuda")
    cuts = [0, 1, 12345, 12345, (1 << 21) + 3, n]  # an empty batch, a one-key batch, batches on both regimes
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        ds.histogram_accumulate(dk[lo:hi], U, H)
    H_ref, _ = oracle.histogram(keys, U)
    np.testing.assert_array_equal(u32(H), H_ref)
    assert ds.stream_status() == ds.OK
    ds.histogram_accumulate(dk, U, H)  # once more: every count doubles
    np.testing.assert_array_equal(u32(H), 2 * H_ref)
