"""Served form: requests that overlap on the device give the same result as alone (bit-exact) and
as the oracle; admission respects the HBM budget; the device loop leaves when idle and comes back."""
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


def dev(a):
    view = a.view(np.int32) if a.dtype == np.uint32 else a.view(np.int16)
    return torch.from_numpy(view.copy()).cuda()


def mixed_requests(count, stream):
    ns = gen.loguniform(count, 6, 20, stream=stream)
    us = gen.loguniform(count, 1, 22, stream=stream + 1)
    w = gen.words(count, stream=stream + 2)
    reqs = []
    for i in range(count):
        width = 2 if w[i] & 1 else 4
        U = int(min(us[i], 65536)) if width == 2 else int(us[i])
        dist = "zipf" if (w[i] >> 1) & 1 else "uniform"
        kind = "sort" if (w[i] >> 2) & 1 else "histogram"
        keys = gen.keys(int(ns[i]), U, dist, width=width, stream=5000 + stream * 1000 + i)
        reqs.append((keys, U, kind))
    return reqs


def test_results_in_the_mix_equal_results_alone(ds):
    reqs = mixed_requests(60, 90)
    srv = ds.Server(hbm_budget_bytes=2 << 30, max_slots=16)
    dkeys = [dev(k) for k, _, _ in reqs]
    tickets = [srv.submit(dk, U, kind) for dk, (_, U, kind) in zip(dkeys, reqs)]  # all at once: they overlap
    for t, dk, (k, U, kind) in zip(tickets, dkeys, reqs):
        res = srv.wait(t)
        assert res["status"] == ds.OK
        H_ref, _ = oracle.histogram(k, U)
        np.testing.assert_array_equal(res["H"].cpu().numpy().view(np.uint32), H_ref)
        if kind == "sort":
            alone = ds.sort(dk, U)  # the same request run alone
            assert torch.equal(res["out"], alone)
            np.testing.assert_array_equal(res["out"].cpu().numpy().view(k.dtype),
                                          oracle.reconstruct(H_ref, U, width=k.dtype.itemsize))
        else:
            alone = ds.histogram(dk, U)
            assert torch.equal(res["H"], alone)
        srv.release(t)
    srv.close()


def test_admission_waits_for_budget(ds):
    # each request needs ~4 MB of H + 4 MB of output + 2 MB of two-level scratch (16-bit low parts); a
    # 12 MB budget admits one at a time
    keys = [dev(gen.keys(1 << 20, 1 << 20, "uniform", stream=95 + i)) for i in range(6)]
    srv = ds.Server(hbm_budget_bytes=12 << 20, max_slots=8)
    ts = [srv.submit(k, 1 << 20, "sort") for k in keys]
    for t, k in zip(ts, keys):
        res = srv.wait(t)
        assert res["status"] == ds.OK
        assert torch.equal(res["out"], torch.sort(k).values)
        srv.release(t)  # frees the arena space the next request is waiting for
    with pytest.raises(ds.DialSortError) as e:
        srv.submit(dev(gen.keys(1 << 22, 1 << 20, "uniform", stream=99)), 1 << 20, "sort")  # 16 MB out alone
    assert e.value.status == ds.ERR_BUDGET
    srv.close()


def test_device_loop_leaves_when_idle_and_comes_back(ds):
    srv = ds.Server(hbm_budget_bytes=64 << 20, max_slots=4, idle_timeout_ns=2_000_000)  # 2 ms
    k = dev(gen.keys(100_000, 5000, "zipf", stream=101))
    for _ in range(3):
        t = srv.submit(k, 5000, "sort")
        res = srv.wait(t)
        assert res["status"] == ds.OK and torch.equal(res["out"], torch.sort(k).values)
        srv.release(t)
        time.sleep(0.03)  # well past the idle timeout: the loop has left and is relaunched
    srv.close()


def test_out_of_range_key_is_reported_per_request(ds):
    srv = ds.Server(hbm_budget_bytes=64 << 20, max_slots=4)
    good = gen.keys(50_000, 777, "uniform", stream=102)
    bad = good.copy()
    bad[123] = 777
    tg = srv.submit(dev(good), 777, "histogram")
    tb = srv.submit(dev(bad), 777, "histogram")
    assert srv.wait(tg)["status"] == ds.OK
    rb = srv.wait(tb)
    assert rb["status"] == ds.ERR_KEY_RANGE
    np.testing.assert_array_equal(rb["H"].cpu().numpy().view(np.uint32), oracle.histogram(bad, 777)[0])
    srv.release(tg)
    srv.release(tb)
    srv.close()
    assert ds.stream_status() == ds.ERR_KEY_RANGE  # the device error word saw it too


@pytest.mark.parametrize("use_server", [True, False])
def test_trace_replay(ds, use_server):
    reqs = mixed_requests(120, 110)
    gaps = -np.log1p(-gen.unit(len(reqs), stream=111)) / 4000.0  # Poisson, 4000 req/s
    arrivals = (np.cumsum(gaps) * 1e9).astype(np.uint64)
    entries = [(dev(k), U, kind, int(t)) for (k, U, kind), t in zip(reqs, arrivals)]
    res, wall = ds.replay(entries, use_server=use_server, hbm_budget_bytes=1 << 30, max_slots=32)
    assert np.all(res["status"] == 0)
    assert np.all(res["done_ns"] >= res["arrival_ns"])
    assert wall >= int(arrivals[-1])
