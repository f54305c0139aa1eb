"""DialSort-Radix (Sec. "Full int32 range") on the GPU: bit-exact against the oracle's four stable
base-256 passes, signed and unsigned, across tile boundaries, ragged tails and skewed digits."""
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


def full_range(n, stream):
    return gen.words(n, stream=stream).astype(np.uint32)


def cases():
    yield "empty", np.zeros(0, dtype=np.uint32)
    yield "one", np.array([0xDEADBEEF], dtype=np.uint32)
    yield "8191", full_range(8191, 9400)
    yield "8192", full_range(8192, 9423)  # one whole tile of 8192 keys
    yield "8193", full_range(8193, 9402)
    yield "tile-1", full_range(16383, 9420)
    yield "tile", full_range(16384, 9401)
    yield "tile+1", full_range(16385, 9421)
    yield "3tiles+5", full_range(3 * 16384 + 5, 9422)
    yield "303tiles+77", full_range(303 * 8192 + 77, 9424)  # more tiles than two CTAs per SM hold at once
    yield "ragged", full_range(1_000_003, 9403)
    yield "zipf-small", gen.keys(2_000_001, 1 << 20, "zipf", stream=9404)  # top two digits all zero
    yield "all-equal", np.full(300_001, 0x80000000, dtype=np.uint32)
    yield "sorted", np.sort(full_range(500_000, 9405))
    yield "reverse", np.sort(full_range(500_000, 9406))[::-1].copy()
    yield "bytes-equal", (full_range(400_000, 9407) & 0xFF00FF00) | 0x00AA0055  # two constant digits


@pytest.mark.parametrize("signed", [True, False])
@pytest.mark.parametrize("name,keys", list(cases()), ids=[c[0] for c in cases()])
def test_radix_matches_oracle(ds, name, keys, signed):
    k = keys.view(np.int32) if signed else keys
    dk = torch.from_numpy(k.view(np.int32)).cuda()
    out = ds.radix_sort(dk, signed=signed)
    torch.cuda.synchronize()
    assert ds.stream_status() == ds.OK
    np.testing.assert_array_equal(out.cpu().numpy().view(k.dtype), oracle.radix_sort(k))


def test_radix_in_place_unaligned_and_host(ds):
    keys = full_range(3_000_000, 9410).view(np.int32)
    ref = oracle.radix_sort(keys)
    dk = torch.from_numpy(keys.copy()).cuda()
    ds.radix_sort(dk, out=dk)  # in place
    np.testing.assert_array_equal(dk.cpu().numpy(), ref)
    big = torch.from_numpy(np.concatenate([np.zeros(1, dtype=np.int32), keys])).cuda()
    sub = big[1:]  # 4-byte but not 16-byte aligned keys
    out = ds.radix_sort(sub)
    np.testing.assert_array_equal(out.cpu().numpy(), ref)
    hk = torch.from_numpy(keys.copy()).pin_memory()
    ho = ds.radix_sort(hk)  # pinned host keys and output
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ho.numpy(), ref)


def test_radix_full_size(ds):
    """2^28 full-range int32 keys, the size the benchmark times: equal to the oracle element by element."""
    n = 1 << 28
    keys = full_range(n, 9411).view(np.int32)
    dk = torch.from_numpy(keys).cuda()
    out = ds.radix_sort(dk)
    torch.cuda.synchronize()
    assert ds.stream_status() == ds.OK
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.radix_sort(keys))
