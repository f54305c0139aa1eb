"""Full-size workloads through the C ABI, compared with the CPU oracle element by element.

* n = 2^28 uint32 keys, U = 2^20: uniform, Zipf s=1.2, all equal, sorted, reverse, sorted runs.
* n = 2^27 uint32 keys, U in {2^8, 2^12, 2^16, 2^20, 2^24, 2^26}, uniform and Zipf s=1.1;
  plus uint16 keys with U = 2^16.
The launch configuration is the library's automatic one, the same the benchmark times.
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


def run_and_compare(ds, keys, U):
    t = torch.from_numpy(keys.view(np.int32 if keys.dtype == np.uint32 else np.int16)).cuda()
    out, H = ds.sort(t, U, return_histogram=True)
    assert ds.stream_status() == ds.OK
    del t
    H_ref, skipped = oracle.histogram(keys, U)
    assert skipped == 0
    np.testing.assert_array_equal(H.cpu().numpy().view(np.uint32), H_ref)
    got = out.cpu().numpy().view(keys.dtype)
    del out
    ref = oracle.reconstruct(H_ref, U, width=keys.dtype.itemsize)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("dist", ["uniform", "zipf", "all_equal", "sorted", "reverse", "runs"])
def test_scale_2p28_keys_u2p20(ds, dist):
    keys = gen.keys(1 << 28, 1 << 20, dist, param=1.2 if dist == "zipf" else None, stream=2 * 16 + 1)
    run_and_compare(ds, keys, 1 << 20)


@pytest.mark.parametrize("logU", [8, 12, 16, 20, 24, 26])
@pytest.mark.parametrize("dist", ["uniform", "zipf"])
def test_universe_sweep_2p27_keys(ds, logU, dist):
    keys = gen.keys(1 << 27, 1 << logU, dist, param=1.1 if dist == "zipf" else None, stream=3 * 16 + logU)
    run_and_compare(ds, keys, 1 << logU)


def test_universe_sweep_u16_keys(ds):
    keys = gen.keys(1 << 27, 1 << 16, "uniform", width=2, stream=3 * 16 + 1)
    run_and_compare(ds, keys, 1 << 16)
