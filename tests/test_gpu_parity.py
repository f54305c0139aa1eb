"""GPU path (through the C ABI) against the CPU oracle: bit-exact, integer work has no tolerance."""
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


def dev(a: np.ndarray, offset: int = 0):
    """Copy a uint32/uint16 array to the GPU, optionally starting `offset` elements into a larger buffer."""
    view = a.view(np.int32) if a.dtype == np.uint32 else a.view(np.int16)
    buf = torch.empty(a.size + offset + 8, dtype=torch.int32 if a.dtype == np.uint32 else torch.int16, device="cuda")
    t = buf[offset:offset + a.size]
    t.copy_(torch.from_numpy(view.copy()))
    return t


def host(t, dtype=np.uint32):
    return t.cpu().numpy().view(dtype)


def check_hist(ds, keys, U, config=None, offset=0, expect_status=0):
    H = ds.histogram(dev(keys, offset), U, config=config)
    st = ds.stream_status()
    H_ref, skipped = oracle.histogram(keys, U)
    assert st == (ds.ERR_KEY_RANGE if skipped else expect_status)
    np.testing.assert_array_equal(host(H), H_ref)
    return H_ref


REGIME_CASES = [
    ("smem32", 256), ("smem32", 4096), ("smem32", 12289),
    ("smem16", 4097), ("smem16", 65536),
    ("global_crn", 65536), ("global_crn", 1 << 20), ("global", 1 << 20), ("global", 7),
]
DISTS = ["uniform", "zipf", "all_equal", "sorted", "runs", "paper_skew", "zipf_perm"]


@pytest.mark.parametrize("regime,U", REGIME_CASES)
@pytest.mark.parametrize("crn", [True, False, "adaptive"])
@pytest.mark.parametrize("width", [4, 2])
@pytest.mark.parametrize("dist", DISTS)
def test_histogram_every_regime(ds, regime, U, crn, width, dist):
    if width == 2 and U > 65536:
        pytest.skip("u16 keys need U <= 65536")
    n = (1 << 18) + 13
    keys = gen.keys(n, U, dist, width=width, param=1000 if dist == "runs" else None, stream=21)
    check_hist(ds, keys, U, config={"regime": regime, "crn": crn})


@pytest.mark.parametrize("n", [0, 1, 31, 32, 33, 1023, 1025, (1 << 16) - 1, (1 << 16) + 1])
@pytest.mark.parametrize("U", [1, 2, 256, 65537])
@pytest.mark.parametrize("offset", [0, 1, 3])
def test_histogram_edge_sizes_and_unaligned_keys(ds, n, U, offset):
    keys = gen.keys(n, U, "uniform", stream=22)
    check_hist(ds, keys, U, offset=offset)
    keys16 = gen.keys(n, min(U, 65536), "zipf", width=2, stream=22)
    check_hist(ds, keys16, min(U, 65536), offset=offset)


@pytest.mark.parametrize("key", ["zero", "last"])
@pytest.mark.parametrize("U", [1 << 16, (1 << 16) - 3, 1 << 20])
def test_all_keys_at_universe_ends(ds, key, U):
    n = (1 << 20) + 3
    keys = np.full(n, 0 if key == "zero" else U - 1, dtype=np.uint32)
    check_hist(ds, keys, U)
    out = ds.sort(dev(keys), U)
    assert ds.stream_status() == ds.OK
    np.testing.assert_array_equal(host(out), keys)


# ---- two-level ingestion (large universes): partition by high bits, count low bits per bucket

TWO_LEVEL_DISTS = ["uniform", "zipf", "all_equal", "sorted", "runs", "paper_skew", "zipf_perm", "reverse"]


@pytest.mark.parametrize("U", [(1 << 17) + 3, 1 << 20, (1 << 22) - 1, (1 << 24) + 5])
@pytest.mark.parametrize("dist", TWO_LEVEL_DISTS)
@pytest.mark.parametrize("crn", ["adaptive", False, True])
def test_two_level_regime(ds, U, dist, crn):
    n = (1 << 20) + 8192 * 3 + 13  # ragged last tile
    keys = gen.keys(n, U, dist, param=5000 if dist == "runs" else None, stream=31)
    H = ds.histogram(dev(keys), U, config={"regime": "two_level", "crn": crn})
    assert ds.stream_status() == ds.OK
    np.testing.assert_array_equal(host(H), oracle.histogram(keys, U)[0])


@pytest.mark.parametrize("n", [3 * (1 << 20) + 5, (1 << 22) + 13, 3_811_443])
@pytest.mark.parametrize("U", [65537, 71454, 84014, 105469, (1 << 17) + 3, 1 << 21])
@pytest.mark.parametrize("dist", ["uniform", "zipf", "all_equal", "sorted"])
def test_two_level_buckets_shared_by_many_count_ctas(ds, n, U, dist):
    """Few buckets, many pass-2 CTAs: buckets counted by several CTAs at once (their histograms merged
    from per-CTA scratch) next to buckets counted by one, in every combination the split produces."""
    keys = gen.keys(n, U, dist, stream=34)
    H = ds.histogram(dev(keys), U, config={"regime": "two_level"})
    assert ds.stream_status() == ds.OK
    np.testing.assert_array_equal(host(H), oracle.histogram(keys, U)[0])


def test_two_level_out_of_range_and_needs_workspace(ds):
    U = 1 << 20
    keys = gen.keys((1 << 20) + 77, U, "uniform", stream=32)
    keys[5] = U
    keys[-3] = 0xFFFFFFFF
    H = ds.histogram(dev(keys), U, config={"regime": "two_level"})
    assert ds.stream_status() == ds.ERR_KEY_RANGE
    np.testing.assert_array_equal(host(H), oracle.histogram(keys, U)[0])
    with pytest.raises(ds.DialSortError) as e:  # forced without a workspace
        ds.histogram(dev(keys[:1000]), U, config={"regime": "two_level"}, use_workspace=False)
    assert e.value.status in (ds.ERR_WORKSPACE, ds.ERR_INVALID_ARG)
    ds.stream_status()


@pytest.mark.parametrize("dist", ["uniform", "zipf", "all_equal"])
def test_sort_uses_two_level_for_large_universe(ds, dist):
    n, U = (1 << 22) + 5, 1 << 21
    keys = gen.keys(n, U, dist, stream=33)
    out, H = ds.sort(dev(keys), U, return_histogram=True)
    assert ds.stream_status() == ds.OK
    H_ref, _ = oracle.histogram(keys, U)
    np.testing.assert_array_equal(host(H), H_ref)
    np.testing.assert_array_equal(host(out), oracle.reconstruct(H_ref, U))


# ---- packed 16-bit counters: carries out of a field are moved to H exactly

@pytest.mark.parametrize("U", [64, 63, 4097])
@pytest.mark.parametrize("pattern", ["low_bin", "high_bin", "last_bin", "pair", "zipf"])
@pytest.mark.parametrize("crn", [True, False, "adaptive"])
def test_smem16_carry_accounting(ds, U, pattern, crn):
    n = (1 << 19) + 7  # one CTA: every bin below would overflow 16 bits several times
    if pattern == "low_bin":
        keys = np.full(n, 2, dtype=np.uint32)
    elif pattern == "high_bin":
        keys = np.full(n, 3, dtype=np.uint32)
    elif pattern == "last_bin":
        keys = np.full(n, U - 1, dtype=np.uint32)  # odd U: the word's high field belongs to no bin
    elif pattern == "pair":
        # bins 4 and 5 share a word and both overflow; the mix makes low carries and word wraps interleave
        r = gen.keys(n, 3, "uniform", stream=23)
        keys = np.where(r == 0, 5, 4).astype(np.uint32)
    else:
        keys = gen.keys(n, U, "zipf", param=1.5, stream=23)
    cfg = {"regime": "smem16", "crn": crn, "blocks": 1, "threads": 256, "replicas": 1}
    check_hist(ds, keys, U, config=cfg)


@pytest.mark.parametrize("regime", ["smem32", "smem16", "global_crn", "global"])
def test_out_of_range_keys_are_reported_and_not_counted(ds, regime):
    U = 1000
    keys = gen.keys((1 << 16) + 5, U, "uniform", stream=24)
    keys[::977] = np.uint32(U + 5)
    keys[1] = np.uint32(0xFFFFFFFF)
    keys[-1] = np.uint32(U)
    check_hist(ds, keys, U, config={"regime": regime})


def test_status_word_is_cleared_after_read(ds):
    keys = np.array([1, 2, 99], dtype=np.uint32)
    ds.histogram(dev(keys), 10)
    assert ds.stream_status() == ds.ERR_KEY_RANGE
    assert ds.stream_status() == ds.OK


# ---- step 2: offsets and projection

def random_hist(U, n, dist, stream):
    keys = gen.keys(n, U, dist, stream=stream)
    H, _ = oracle.histogram(keys, U)
    return H


@pytest.mark.parametrize("U", [1, 3, 1000, 1024, 1025, 4096 + 7, 1 << 20])
@pytest.mark.parametrize("dist", ["uniform", "zipf", "all_equal", "sorted"])
def test_offsets_match_oracle(ds, U, dist):
    n = 300_007
    H = random_hist(U, n, dist, 25)
    O = ds.offsets(dev(H), U, n).cpu().numpy().astype(np.uint64)
    ref = oracle.offsets(H, U)
    chunks = (U + 1023) // 1024
    np.testing.assert_array_equal(O[:chunks], ref[np.arange(chunks) * 1024])
    assert int(O[chunks]) == n == int(ref[U])


@pytest.mark.parametrize("U", [1, 3, 1000, 1025, 4096 + 7, 65536, 1 << 20, 1 << 24])
@pytest.mark.parametrize("dist", ["uniform", "zipf", "all_equal", "paper_skew"])
@pytest.mark.parametrize("n", [1, 8191, 8192, 8193, 300_007])
def test_reconstruct_matches_oracle(ds, U, dist, n):
    H = random_hist(U, n, dist, 26)
    out = ds.reconstruct(dev(H), U, n)
    assert ds.stream_status() == ds.OK
    np.testing.assert_array_equal(host(out), oracle.reconstruct(H, U))


@pytest.mark.parametrize("U,width", [(1 << 22, 4), ((1 << 20) + 9, 4), (65536, 2), (3 * 1024 + 5, 4)])
@pytest.mark.parametrize("cap_kind", ["exact", "larger", "smaller"])
def test_sparse_projection_short_and_long_runs(ds, U, width, cap_kind):
    # fewer keys than bins / 4: the bin-parallel projection; bins holding 1-4 keys (a lane writes them),
    # 5-300 keys and one bin of many keys (the warp paints them), spread over the universe
    rng = np.random.default_rng(U + width)
    H = np.zeros(U, dtype=np.uint32)
    nz = rng.choice(U, size=max(1, U // 40), replace=False)
    H[nz] = rng.integers(1, 5, size=nz.size)
    mid = rng.choice(U, size=max(1, U // 2000), replace=False)
    H[mid] = rng.integers(5, 300, size=mid.size)
    H[rng.integers(0, U)] += U // 16
    n = int(H.sum())
    cap = {"exact": n, "larger": n + n // 8, "smaller": n - n // 2}[cap_kind]
    assert 4 * cap < U
    fill = 0xBEEF if width == 2 else 0xDEADBEEF
    out = dev(np.full(cap, fill, dtype=np.uint16 if width == 2 else np.uint32))
    ds.reconstruct(dev(H), U, cap, out=out)
    assert ds.stream_status() == (ds.ERR_OVERFLOW if cap < n else ds.OK)
    want = oracle.reconstruct(H, U, width=width)
    got = host(out, np.uint16 if width == 2 else np.uint32)
    np.testing.assert_array_equal(got[:min(cap, n)], want[:min(cap, n)])
    if cap > n:
        assert np.all(got[n:] == fill)  # past sum(H) nothing is written


@pytest.mark.parametrize("U", [1, 300, 65536])
@pytest.mark.parametrize("offset", [0, 1, 5])
def test_reconstruct_u16_and_unaligned_out(ds, U, offset):
    n = 100_003
    H = random_hist(U, n, "zipf", 27)
    out = dev(np.zeros(n, dtype=np.uint16), offset)
    ds.reconstruct(dev(H), U, n, out=out)
    assert ds.stream_status() == ds.OK
    np.testing.assert_array_equal(host(out, np.uint16), oracle.reconstruct(H, U, width=2))
    out32 = dev(np.zeros(n, dtype=np.uint32), offset)
    ds.reconstruct(dev(H), U, n, out=out32)
    np.testing.assert_array_equal(host(out32), oracle.reconstruct(H, U))


def test_reconstruct_capacity_larger_and_smaller_than_sum(ds):
    U, n = 5000, 50_000
    H = random_hist(U, n, "uniform", 28)
    ref = oracle.reconstruct(H, U)
    big = dev(np.full(n + 777, 0xDEADBEEF, dtype=np.uint32))
    ds.reconstruct(dev(H), U, n + 777, out=big)
    assert ds.stream_status() == ds.OK
    got = host(big)
    np.testing.assert_array_equal(got[:n], ref)
    assert np.all(got[n:] == 0xDEADBEEF)  # past sum(H) nothing is written
    small = dev(np.full(n - 1000, 7, dtype=np.uint32))
    ds.reconstruct(dev(H), U, n - 1000, out=small)
    assert ds.stream_status() == ds.ERR_OVERFLOW
    np.testing.assert_array_equal(host(small), ref[: n - 1000])


def test_reconstruct_empty_histogram(ds):
    U = 4096
    out = dev(np.full(100, 9, dtype=np.uint32))
    ds.reconstruct(dev(np.zeros(U, dtype=np.uint32)), U, 100, out=out)
    assert ds.stream_status() == ds.OK
    assert np.all(host(out) == 9)


# ---- both steps

@pytest.mark.parametrize("dist", ["uniform", "zipf", "all_equal", "reverse", "runs"])
@pytest.mark.parametrize("width", [4, 2])
def test_sort_in_place(ds, dist, width):
    n, U = (1 << 20) + 5, 1 << 16
    keys = gen.keys(n, U, dist, width=width, param=1 << 14 if dist == "runs" else None, stream=29)
    t = dev(keys, 1)
    ds.sort(t, U, out=t)
    assert ds.stream_status() == ds.OK
    np.testing.assert_array_equal(host(t, keys.dtype), oracle.sort(keys, U))


def test_small_uniform_workload(ds):
    """n = 2^20 uint32 keys uniform on [0, 2^16): histogram and sorted output."""
    n, U = 1 << 20, 1 << 16
    keys = gen.keys(n, U, "uniform", stream=1)
    out, H = ds.sort(dev(keys), U, return_histogram=True)
    assert ds.stream_status() == ds.OK
    H_ref, _ = oracle.histogram(keys, U)
    np.testing.assert_array_equal(host(H), H_ref)
    np.testing.assert_array_equal(host(out), oracle.reconstruct(H_ref, U))


def test_deterministic_repeat(ds):
    n, U = 1 << 20, 1 << 20
    keys = dev(gen.keys(n, U, "zipf", stream=30))
    a = host(ds.sort(keys, U)).copy()
    b = host(ds.sort(keys, U))
    np.testing.assert_array_equal(a, b)
