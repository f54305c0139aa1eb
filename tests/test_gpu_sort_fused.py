"""The two-level sort with counting fused into the projection (pass 2 and Eq. (2) in one persistent
kernel), against the CPU oracle element by element: the sorted output and the histogram the sort leaves
in its workspace.  The planner runs without a measured table here, so every shape below takes the
two-level form (2^16 < U <= 2^21, n >= 2^20, 16-byte aligned uint32 keys)."""
import os

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

    ds.tune_table_load(None)
    assert ds.stream_status() == ds.OK
    yield ds
    ds.tune_table_load(ds.TUNE_TABLE if os.path.exists(ds.TUNE_TABLE) else None)


def dev(a: np.ndarray, offset: int = 0):
    buf = torch.empty(a.size + offset + 8, dtype=torch.int32, device="cuda")
    t = buf[offset:offset + a.size]
    t.copy_(torch.from_numpy(a.view(np.int32)))
    return t


def host(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("n", [1 << 20, 3 * (1 << 20) + 5, (1 << 22) + 13, 3_811_443])
@pytest.mark.parametrize("U", [65537, 71454, 105469, (1 << 17) + 3, 1 << 20, (1 << 21) - 5, 1 << 21])
@pytest.mark.parametrize("dist", ["uniform", "zipf", "all_equal", "sorted", "runs"])
def test_fused_sort_matches_oracle(ds, n, U, dist):
    keys = gen.keys(n, U, dist, param=4096 if dist == "runs" else None, stream=81)
    assert ds.plan_histogram(n, U)["regime_name"] == "two_level"
    out, H = ds.sort(dev(keys), U, return_histogram=True)
    assert ds.stream_status() == ds.OK
    H_ref, skipped = oracle.histogram(keys, U)
    assert skipped == 0
    np.testing.assert_array_equal(host(H), H_ref)
    np.testing.assert_array_equal(host(out), oracle.reconstruct(H_ref, U))


@pytest.mark.parametrize("U", [1 << 18, (1 << 20) + 3])
def test_fused_sort_in_place_and_unaligned_output(ds, U):
    n = 2 * (1 << 20) + 9
    keys = gen.keys(n, U, "zipf", stream=82)
    want = oracle.sort(keys, U)
    k = dev(keys)
    ds.sort(k, U, out=k)  # in place
    assert ds.stream_status() == ds.OK
    np.testing.assert_array_equal(host(k), want)
    out = dev(np.zeros(n, dtype=np.uint32), offset=1)  # 4-byte aligned only: scalar stores at the run ends
    ds.sort(dev(keys), U, out=out)
    assert ds.stream_status() == ds.OK
    np.testing.assert_array_equal(host(out), want)


def test_fused_sort_keys_out_of_range(ds):
    U = 1 << 20
    keys = gen.keys((1 << 21) + 3, U, "uniform", stream=83)
    keys[7] = U
    keys[-1] = 0xFFFFFFFF
    out = dev(np.full(keys.size, 0xDEADBEEF, dtype=np.uint32))
    ds.sort(dev(keys), U, out=out)
    assert ds.stream_status() == ds.ERR_KEY_RANGE
    H_ref, skipped = oracle.histogram(keys, U)
    assert skipped == 2
    got = host(out)
    np.testing.assert_array_equal(got[:-2], oracle.reconstruct(H_ref, U))  # the kept keys, in order
    assert np.all(got[-2:] == 0xDEADBEEF)  # past sum(H) nothing is written


def test_fused_sort_repeated_calls_share_a_workspace(ds):
    U = (1 << 19) + 1
    ws = torch.empty(ds.sort_workspace_size(1 << 21, U), dtype=torch.uint8, device="cuda")
    for i, dist in enumerate(["uniform", "all_equal", "zipf", "sorted"]):
        keys = gen.keys((1 << 21) - 3 * i, U, dist, stream=84 + i)
        out = ds.sort(dev(keys), U, ws=ws)
        assert ds.stream_status() == ds.OK
        np.testing.assert_array_equal(host(out), oracle.sort(keys, U))
