"""Mapped-domain sort (Prop. "General Self-Indexing Principle") on the GPU: keys counted at phi(key)
and emitted as phi_inv(index), bit-exact against the oracle, for 8-, 16- and 32-bit raw keys."""
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


def cuda(a):
    a = np.ascontiguousarray(a)
    view = {1: np.uint8, 2: np.int16, 4: np.int32}[a.dtype.itemsize]
    return torch.from_numpy(a.view(view)).cuda()


def host(t, dtype):
    return t.cpu().numpy().view(dtype)


@pytest.mark.parametrize("n", [1, 15, 17, (1 << 22) + 3])
@pytest.mark.parametrize("dist", ["uniform", "zipf", "all_equal"])
def test_pixels_identity_u8(ds, n, dist):
    px = gen.keys(n, 256, dist, stream=9600 + n % 7).astype(np.uint8)
    out = ds.sort_mapped(cuda(px), 256)
    assert ds.stream_status() == ds.OK
    np.testing.assert_array_equal(host(out, np.uint8), oracle.sort_mapped(px, 256)[0])


def rank_maps(S, M):
    phi = np.full(M, 0xFFFFFFFF, dtype=np.uint32)
    phi[S] = np.arange(S.size, dtype=np.uint32)
    return phi


@pytest.mark.parametrize("width,M,size", [(2, 65536, 5000), (4, 1 << 24, 4096), (4, 1 << 24, 60_000)])
def test_sparse_domain_through_rank_maps(ds, width, M, size):
    S = np.unique(gen.keys(size + size // 8, M, "uniform", stream=9700 + size))[:size]
    phi = rank_maps(S, M)
    dt = np.uint16 if width == 2 else np.uint32
    keys = S[gen.keys(3_000_001, S.size, "zipf", stream=9701)].astype(dt)
    out = ds.sort_mapped(cuda(keys), S.size, phi=cuda(phi), phi_inv=cuda(S.astype(dt)))
    assert ds.stream_status() == ds.OK
    ref, _, skipped = oracle.sort_mapped(keys, S.size, phi, S)
    assert skipped == 0
    np.testing.assert_array_equal(host(out, dt), ref)


def test_keys_outside_the_domain_are_reported(ds):
    S = np.arange(0, 2000, 2, dtype=np.uint32)  # even values only
    M = 2000
    phi = rank_maps(S, M)
    keys = S[gen.keys(100_000, S.size, "uniform", stream=9702)]
    keys[[5, 500, 50_000]] = [3, 1999, 5000]  # odd values and one beyond M: outside the domain
    out = torch.zeros(keys.size, dtype=torch.int32, device="cuda")
    ds.sort_mapped(cuda(keys), S.size, phi=cuda(phi), phi_inv=cuda(S), out=out)
    assert ds.stream_status() == ds.ERR_KEY_RANGE
    ref, _, skipped = oracle.sort_mapped(keys, S.size, phi, S)
    assert skipped == 3
    np.testing.assert_array_equal(host(out, np.uint32)[: ref.size], ref)


def test_in_place_and_reverse_order(ds):
    U = 3000
    phi = (U - 1 - np.arange(U)).astype(np.uint32)  # reverses the domain; its own inverse
    keys = gen.keys((1 << 20) + 9, U, "zipf", stream=9703)
    d = cuda(keys)
    ds.sort_mapped(d, U, phi=cuda(phi), phi_inv=cuda(phi), out=d)
    np.testing.assert_array_equal(host(d, np.uint32), oracle.sort_mapped(keys, U, phi, phi)[0])
