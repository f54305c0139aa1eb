"""Batched form: many uneven instances in one persistent launch, each bit-exact against the oracle
and against the same instance run alone through the single-instance entry points."""
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


def dev(a, offset=0):
    view = a.view(np.int32) if a.dtype == np.uint32 else a.view(np.int16)
    buf = torch.empty(a.size + offset + 8, dtype=torch.int32 if a.dtype == np.uint32 else torch.int16, device="cuda")
    t = buf[offset:offset + a.size]
    t.copy_(torch.from_numpy(view.copy()))
    return t


def host(t, dtype):
    return t.cpu().numpy().view(dtype)


def make_instances(count, seed_stream, n_lo=4, n_hi=18, u_lo=1, u_hi=20, with_u16=True):
    ns = gen.loguniform(count, n_lo, n_hi, stream=seed_stream)
    us = gen.loguniform(count, u_lo, u_hi, stream=seed_stream + 1)
    picks = gen.words(count, stream=seed_stream + 2)
    inst = []
    for i in range(count):
        n, U = int(ns[i]), int(us[i])
        width = 2 if (with_u16 and picks[i] % 4 == 0) else 4
        if width == 2:
            U = min(U, 65536)
        dist = ["uniform", "zipf", "all_equal"][int(picks[i] >> 8) % 3]
        keys = gen.keys(n, U, dist, width=width, stream=1000 + seed_stream * 8192 + i)
        inst.append((keys, U))
    # edge cases: empty, U = 1, a single key, unaligned keys
    inst.append((np.zeros(0, dtype=np.uint32), 17))
    inst.append((np.zeros(5000, dtype=np.uint32), 1))
    inst.append((np.array([6], dtype=np.uint32), 7))
    inst.append((gen.keys(12345, 999, "uniform", stream=7), 999))
    return inst


@pytest.mark.parametrize("sort", [True, False])
def test_batch_matches_oracle_and_single_runs(ds, sort):
    inst = make_instances(96, 50)
    offsets = [(i % 3) for i in range(len(inst))]  # unaligned starts for a third of the instances
    keys = [dev(k, o) for (k, _), o in zip(inst, offsets)]
    U = [u for _, u in inst]
    b = ds.Batch(keys, U, sort=sort).launch()
    torch.cuda.synchronize()
    assert ds.stream_status() == ds.OK
    for i, (k, u) in enumerate(inst):
        H_ref, _ = oracle.histogram(k, u)
        np.testing.assert_array_equal(host(b.H[i], np.uint32), H_ref, err_msg=f"instance {i} n={k.size} U={u}")
        if sort:
            np.testing.assert_array_equal(host(b.out[i], k.dtype), oracle.reconstruct(H_ref, u, width=k.dtype.itemsize))
            alone = ds.sort(keys[i], u)  # the same instance through the single-instance path
            assert torch.equal(alone, b.out[i])
    b.close()


def test_batch_relaunch_and_plan_description(ds):
    inst = make_instances(40, 60, with_u16=False)
    keys = [dev(k) for k, _ in inst]
    U = [u for _, u in inst]
    b = ds.Batch(keys, U, sort=True)
    for _ in range(3):  # the plan tables are re-uploaded each launch; results identical
        for h in b.H:
            h.fill_(-1)
        b.launch()
        torch.cuda.synchronize()
        assert ds.stream_status() == ds.OK
        for i, (k, u) in enumerate(inst):
            np.testing.assert_array_equal(host(b.out[i], np.uint32), np.sort(k))
    regimes = {b.describe(i)["regime_name"] for i in range(len(inst))}
    assert regimes <= {"smem32", "smem16", "global_crn", "two_level"}
    b.close()


TWO_LEVEL_CASES = [  # (n, U, dist, width, offset): universes past the packed sub-histogram, up to 2^22 bins
    (13_000, 24_577, "uniform", 4, 0), (12_289, 24_577, "zipf", 4, 1), (40_000, 65536, "uniform", 2, 0),
    (6 * 8192 + 5, 65536, "all_equal", 2, 3), (3 * 8192 + 5, 40000, "sorted", 4, 2),
    ((1 << 20) + 77, 100003, "zipf", 4, 0), ((1 << 20) + 77, 1 << 20, "uniform", 4, 1),
    (3 << 20, 3 * (1 << 20) + 1, "uniform", 4, 0), ((1 << 21) + 13, 1 << 22, "zipf", 4, 0),
    ((1 << 21) + 13, 1 << 22, "all_equal", 4, 2), (5_000_003, 300_007, "runs", 4, 0),
    (2_000_001, 1 << 21, "sorted", 4, 0), (40_000, 65535, "zipf_perm", 2, 1),
]


@pytest.mark.parametrize("sort", [True, False])
def test_batch_two_level_instances(ds, sort):
    inst = [(gen.keys(n, U, d, width=w, param=4096 if d == "runs" else None, stream=90 + i), U, o)
            for i, (n, U, d, w, o) in enumerate(TWO_LEVEL_CASES)]
    inst.append((gen.keys(300_000, 256, "uniform", stream=99), 256, 0))  # a small-universe neighbour
    keys = [dev(k, o) for k, _, o in inst]
    regimes = ["two_level"] * len(TWO_LEVEL_CASES) + ["auto"]
    b = ds.Batch(keys, [u for _, u, _ in inst], sort=sort, regime=regimes)
    b.launch()
    torch.cuda.synchronize()
    assert ds.stream_status() == ds.OK
    for i, (k, u, _) in enumerate(inst):
        d = b.describe(i)
        if i < len(TWO_LEVEL_CASES):
            assert d["regime_name"] == "two_level", (i, d)
            assert d["items"][1] >= (k.size + 8191) // 8192 + (u + 16383) // 16384  # partition + count items
        H_ref, _ = oracle.histogram(k, u)
        np.testing.assert_array_equal(host(b.H[i], np.uint32), H_ref, err_msg=f"instance {i} n={k.size} U={u}")
        if sort:
            np.testing.assert_array_equal(host(b.out[i], k.dtype), oracle.reconstruct(H_ref, u, width=k.dtype.itemsize),
                                          err_msg=f"instance {i}")
    b.close()


def test_batch_two_level_reports_out_of_range_keys(ds):
    k = gen.keys(100_000, 70_000, "uniform", stream=98)
    bad = k.copy()
    bad[12345] = 70_000
    bad[99_999] = 0xFFFFFFFF
    b = ds.Batch([dev(bad)], [70_000], sort=False, regime="two_level")
    assert b.describe(0)["regime_name"] == "two_level"
    b.launch()
    torch.cuda.synchronize()
    assert ds.stream_status() == ds.ERR_KEY_RANGE
    np.testing.assert_array_equal(host(b.H[0], np.uint32), oracle.histogram(bad, 70_000)[0])
    b.close()


def test_batch_forced_regimes_and_refusals(ds):
    k = gen.keys(200_000, 5000, "zipf", stream=97)
    H_ref, _ = oracle.histogram(k, 5000)
    for regime in ("smem32", "smem16", "global_crn", "global", "two_level"):
        b = ds.Batch([dev(k)], [5000], sort=True, regime=regime)
        assert b.describe(0)["regime_name"] == ("global_crn" if regime == "global" else regime)
        b.launch()
        torch.cuda.synchronize()
        assert ds.stream_status() == ds.OK
        np.testing.assert_array_equal(host(b.H[0], np.uint32), H_ref)
        np.testing.assert_array_equal(host(b.out[0], np.uint32), oracle.reconstruct(H_ref, 5000))
        b.close()
    big = dev(gen.keys(1000, 1 << 23, "uniform", stream=96))
    for regime in ("smem32", "smem16", "two_level", "cluster"):  # too large for these, or not built
        with pytest.raises(ds.DialSortError):
            ds.Batch([big], [1 << 23], sort=True, regime=regime)


def test_batch_captured_in_a_cuda_graph(ds):
    inst = make_instances(48, 70, with_u16=False)
    keys = [dev(k) for k, _ in inst]
    U = [u for _, u in inst]
    b = ds.Batch(keys, U, sort=True)
    b.launch()  # first launch sets up kernel attributes outside the capture
    torch.cuda.synchronize()
    for o in b.out:
        o.zero_()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            b.launch(stream=s)
    torch.cuda.synchronize()
    for o in b.out:
        o.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert ds.stream_status() == ds.OK
    for i, (k, u) in enumerate(inst):
        np.testing.assert_array_equal(host(b.out[i], np.uint32), np.sort(k))
    del g
    b.close()


def test_batch_reports_out_of_range_keys(ds):
    good = gen.keys(10000, 100, "uniform", stream=80)
    bad = good.copy()
    bad[17] = 100
    H, _ = ds.batched([dev(good), dev(bad)], [100, 100], sort=False)
    assert ds.stream_status() == ds.ERR_KEY_RANGE
    np.testing.assert_array_equal(host(H[1], np.uint32), oracle.histogram(bad, 100)[0])


def test_empty_batch(ds):
    H, out = ds.batched([], [], sort=True)
    assert H == [] and out == []
