"""The skew probe and the tuned plans on the device.

* The probe's counts equal the same statistics computed on the host from the same sampled positions
  (dense windows for n <= 4096, 128 spread windows above), for 32- and 16-bit keys, with keys >= U
  mixed in; its classes are the expected ones on the canonical inputs.
* Every launch choice of the shipped tuning table (and of a test table that names every regime), run
  as the planner runs it, gives the oracle's histogram and sorted output, element by element.
* Skew classes fed to the batched engine and to dialsort_sort_ex keep results identical to the oracle.
"""
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

    assert ds.stream_status() == ds.OK
    yield ds
    ds.tune_table_load(ds.TUNE_TABLE if os.path.exists(ds.TUNE_TABLE) else None)


def dev(a: np.ndarray):
    return torch.from_numpy(a.view(np.int32) if a.dtype == np.uint32 else a.view(np.int16)).cuda()


def host_probe(keys: np.ndarray, U: int):
    """The probe's statistics from its sample positions, computed on the host."""
    n = keys.size
    if n <= 4096:
        starts = [32 * w for w in range((n + 31) // 32)]
    else:
        starts = [(n - 32) * w // 127 for w in range(128)]
    samples = eq = pairs = 0
    counts = {}
    for s in starts:
        win = [int(keys[i]) if i < n else None for i in range(s, s + 32)]
        ok = [k is not None and k < U for k in win]
        for j in range(32):
            if ok[j]:
                samples += 1
                counts[win[j]] = counts.get(win[j], 0) + 1
            if j > 0 and ok[j] and ok[j - 1]:
                pairs += 1
                eq += win[j] == win[j - 1]
    return samples, eq, pairs, max(counts.values()) if counts else 0


CASES = [
    (0, 256, "uniform", 4), (1, 256, "uniform", 4), (31, 4096, "all_equal", 4), (33, 7, "uniform", 2),
    (1000, 1 << 16, "zipf", 2), (4096, 1 << 20, "sorted", 4), (4097, 1 << 20, "uniform", 4),
    (100003, 1 << 12, "runs", 4), ((1 << 20) + 5, 1 << 20, "zipf", 4), ((1 << 20) + 5, 1 << 24, "uniform", 4),
    ((1 << 22) + 3, 1 << 16, "sorted", 2), ((1 << 22) + 3, 1000, "paper_skew", 4),
]


@pytest.mark.parametrize("n,U,dist,width", CASES)
def test_probe_counts_match_host(ds, n, U, dist, width):
    keys = gen.keys(n, U, dist, width=width, param=64 if dist == "runs" else None, stream=51)
    if n > 10:  # a few keys outside the universe: not sampled
        keys = keys.copy()
        keys[3] = U if width == 4 or U < 65536 else keys[3]
        keys[n // 2] = U + 5 if width == 4 or U + 5 < 65536 else keys[n // 2]
    r = ds.probe_skew(dev(keys) if n else torch.empty(0, dtype=torch.int32, device="cuda"), U)
    s, eq, pairs, top = host_probe(keys, U)
    assert (r["samples"], r["equal_neighbours"], r["neighbour_pairs"], r["top_multiplicity"]) == (s, eq, pairs, top)
    assert ds.stream_status() == ds.OK  # keys >= U raise nothing in the probe


@pytest.mark.parametrize("dist,U,want", [
    ("uniform", 1 << 20, "low"), ("uniform", 1 << 8, "low"), ("zipf", 1 << 20, "hot"), ("zipf", 1 << 8, "hot"),
    ("sorted", 1 << 12, "runs"), ("all_equal", 1 << 20, "runs"), ("paper_skew", 1 << 16, "low"),
    ("paper_skew", 1 << 8, "hot"),
])
def test_probe_classes(ds, dist, U, want):
    keys = gen.keys((1 << 22) + 1, U, dist, stream=52)
    assert ds.probe_skew(dev(keys), U)["skew_name"] == want


def test_probe_batched_equals_single(ds):
    items = [(70001, 1 << 10, "zipf"), (3, 5, "uniform"), (1 << 20, 1 << 20, "uniform"), (50000, 1 << 16, "sorted"),
             (0, 9, "uniform")]
    ks = [dev(gen.keys(n, U, d, stream=53 + i)) if n else torch.empty(0, dtype=torch.int32, device="cuda")
          for i, (n, U, d) in enumerate(items)]
    b = ds.Batch(ks, [U for _, U, _ in items], sort=True, skew="probe")
    for i, (n, U, _) in enumerate(items):
        want = ds.probe_skew(ks[i], U)["skew_class"] if n else 0
        assert b.skew[i] == want
    b.close()


def _entries(path):
    out = []
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            out.append(tuple(map(int, line.split())))
    return out


TEST_TABLE = """20 8 4 1 1 2 32 1024 1
20 8 4 2 1 3 4 512 2
20 12 4 3 1 1 2 256 4
22 14 4 1 2 2 1 512 0
22 14 4 2 2 3 2 1024 1
22 16 2 3 2 1 1 1024 2
22 20 4 1 5 2 0 512 0
22 20 4 2 4 1 0 256 0
22 22 4 2 4 3 0 1024 2
22 18 4 1 6 0 0 0 0
"""

DIST_OF_SKEW = {0: "uniform", 1: "uniform", 2: "zipf", 3: "sorted"}


def _run_table(ds, path):
    """Each distinct choice of a table, forced as explicit launch fields, and the planner's own plan
    at the entry's shape class, against the oracle."""
    ds.tune_table_load(path)
    sms = ds.lib().dialsort_device_sm_count()
    seen = set()
    for lg_n, lg_u, width, skew, regime, crn, rep, threads, per_sm in _entries(path):
        choice = (regime, crn, rep, threads, per_sm)
        if (choice, width) in seen:
            continue
        seen.add((choice, width))
        n = min(1 << lg_n, (1 << 21) + 77) + 13  # several tiles and a ragged tail
        U = (1 << lg_u) - 3 if regime == 6 else min(1 << lg_u, 1 << 22) - 3
        if width == 2:
            U = min(U, 65536)
        keys = gen.keys(n, U, DIST_OF_SKEW[skew], width=width, stream=54)
        H_ref, skipped = oracle.histogram(keys, U)
        assert skipped == 0
        want = oracle.reconstruct(H_ref, U, width)
        config = None
        if regime:
            config = {"regime": ds.REGIME_NAMES[regime]}
            for k, v in (("crn", crn), ("replicas", rep), ("threads", threads), ("blocks", per_sm * sms)):
                if v:
                    config[k] = v
        for cfg in ([config] if config else []) + [None]:
            H = ds.histogram(dev(keys), U, config=cfg, skew=skew)
            out = ds.sort(dev(keys), U, config=cfg, skew=skew)
            assert ds.stream_status() == ds.OK, (choice, cfg)
            np.testing.assert_array_equal(H.cpu().numpy().view(np.uint32), H_ref, err_msg=str((choice, cfg)))
            got = out.cpu().numpy().view(np.uint32 if width == 4 else np.uint16)
            np.testing.assert_array_equal(got, want, err_msg=str((choice, cfg)))
    return seen


def test_every_regime_a_table_can_name(ds, tmp_path):
    p = tmp_path / "t.txt"
    p.write_text(TEST_TABLE)
    seen = _run_table(ds, str(p))
    assert len(seen) == len(TEST_TABLE.strip().splitlines())


def test_shipped_table_choices(ds):
    if not os.path.exists(ds.TUNE_TABLE):
        pytest.skip("no measured table shipped")
    _run_table(ds, ds.TUNE_TABLE)


@pytest.mark.parametrize("skew", ["low", "hot", "runs"])
def test_batched_engine_with_skew_classes(ds, skew):
    rng_items = [(200003, 1 << 8), (65536, 1 << 14), (1 << 20, 1 << 18), (3001, 1 << 20), (77, 3)]
    dist = {"low": "uniform", "hot": "zipf", "runs": "sorted"}[skew]
    host_keys = [gen.keys(n, U, dist, stream=55 + i) for i, (n, U) in enumerate(rng_items)]
    b = ds.Batch([dev(k) for k in host_keys], [U for _, U in rng_items], sort=True, skew=[skew] * len(rng_items))
    b.launch()
    torch.cuda.synchronize()
    assert ds.stream_status() == ds.OK
    for i, (n, U) in enumerate(rng_items):
        d = b.describe(i)
        assert d["skew"] == skew
        if skew == "low":
            assert d["crn"] in ("off", "on", "adaptive")
        H_ref, _ = oracle.histogram(host_keys[i], U)
        np.testing.assert_array_equal(b.H[i].cpu().numpy().view(np.uint32), H_ref)
        np.testing.assert_array_equal(b.out[i].cpu().numpy().view(np.uint32), oracle.reconstruct(H_ref, U))
    b.close()


def test_served_requests_with_skew_classes(ds):
    srv = ds.Server(hbm_budget_bytes=1 << 30, max_slots=8)
    cases = [(300007, 1 << 12, "zipf", "hot"), (100000, 1 << 16, "uniform", "low"), (50000, 1 << 8, "sorted", "runs")]
    ks = [gen.keys(n, U, d, stream=60 + i) for i, (n, U, d, _) in enumerate(cases)]
    tickets = [srv.submit(dev(k), U, "sort", skew=s) for k, (_, U, _, s) in zip(ks, cases)]
    for t, k, (n, U, _, _) in zip(tickets, ks, cases):
        res = srv.wait(t)
        assert res["status"] == ds.OK
        H_ref, _ = oracle.histogram(k, U)
        np.testing.assert_array_equal(res["H"].cpu().numpy().view(np.uint32), H_ref)
        np.testing.assert_array_equal(res["out"].cpu().numpy().view(np.uint32), oracle.reconstruct(H_ref, U))
        srv.release(t)
    srv.close()
