"""The batched and served configurations at full size, every result against the CPU oracle.

* Batched: the benchmark's own 4096 instances (n_i log-uniform in [2^10, 2^22], U_i log-uniform in
  [2^8, 2^20], uniform / Zipf 1.2 / all equal; about 2.1e9 keys) in one persistent launch; every
  instance's histogram and sorted output compared with oracle.histogram / oracle.reconstruct, element
  by element.
* Served: the first 2000 requests of the benchmark's Poisson trace (n log-uniform in [2^12, 2^26], U
  log-uniform in [2^8, 2^24], uint32 and uint16 keys, sort and histogram, uniform and Zipf), all
  submitted at once so that they overlap on the device as slots and arena space free up; every
  histogram compared with the oracle's, every sorted output checked against the oracle's histogram
  (a nondecreasing sequence whose histogram is H is the unique projection of H, Eq. (2)), and every
  result compared with the same request run alone.

The oracle runs on the host cores in threads (its C routines release the interpreter lock) while the
device works.
"""
import concurrent.futures
import os

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


def _align(x, a):
    return (x + a - 1) // a * a


def _workers():
    return max(4, min(32, os.cpu_count() or 4))


def test_batched_configuration_full_size(ds):
    count = 4096
    ns, us, dists = gen.batch_workload(count)
    koff = np.zeros(count + 1, dtype=np.int64)
    hoff = np.zeros(count + 1, dtype=np.int64)
    for i in range(count):
        koff[i + 1] = koff[i] + _align(int(ns[i]), 64)
        hoff[i + 1] = hoff[i] + _align(int(us[i]), 64)
    host = np.empty(int(koff[-1]), dtype=np.uint32)
    with concurrent.futures.ThreadPoolExecutor(max_workers=_workers()) as ex:
        list(ex.map(lambda i: gen.batch_keys(i, ns[i], us[i], dists[i], out=host[koff[i]:koff[i] + ns[i]]),
                    range(count)))
    keys_d = torch.from_numpy(host.view(np.int32)).cuda()
    out_d = torch.full_like(keys_d, -1)
    H_d = torch.full((int(hoff[-1]),), -1, dtype=torch.int32, device="cuda")
    kv = [keys_d[koff[i]:koff[i] + ns[i]] for i in range(count)]
    ov = [out_d[koff[i]:koff[i] + ns[i]] for i in range(count)]
    hv = [H_d[hoff[i]:hoff[i] + us[i]] for i in range(count)]
    b = ds.Batch(kv, [int(u) for u in us], H=hv, out=ov, sort=True)
    b.launch()
    torch.cuda.synchronize()
    assert ds.stream_status() == ds.OK
    b.close()
    Hh = H_d.cpu().numpy().view(np.uint32)
    outh = out_d.cpu().numpy().view(np.uint32)
    del keys_d, out_d, H_d, kv, ov, hv

    def check(i):
        k = host[koff[i]:koff[i] + ns[i]]
        H_ref, skipped = oracle.histogram(k, int(us[i]))
        if skipped:
            return f"instance {i}: the generator drew a key >= U"
        if not np.array_equal(Hh[hoff[i]:hoff[i] + us[i]], H_ref):
            return f"instance {i} (n={ns[i]} U={us[i]} {dists[i]}): histogram differs from the oracle"
        if not np.array_equal(outh[koff[i]:koff[i] + ns[i]], oracle.reconstruct(H_ref, int(us[i]))):
            return f"instance {i} (n={ns[i]} U={us[i]} {dists[i]}): sorted output differs from the oracle"
        return None

    with concurrent.futures.ThreadPoolExecutor(max_workers=_workers()) as ex:
        errors = [e for e in ex.map(check, range(count)) if e]
    assert not errors, errors[:5]


def _unsigned(t):
    return t.to(torch.int32) & 0xFFFF if t.dtype == torch.int16 else t


def test_served_configuration_trace_slice(ds):
    R = 2000
    tr = gen.served_trace()
    pools_host = {(d, w): gen.served_pool(d, w) for d in ("uniform", "zipf") for w in (4, 2)}

    def oracle_hist(i):
        w, c = int(tr["width"][i]), int(tr["cls"][i])
        k = gen.served_request_keys(pools_host[(str(tr["dist"][i]), w)], w, c, int(tr["start"][i]), int(tr["n"][i]))
        H, skipped = oracle.histogram(k, int(tr["U"][i]))
        assert skipped == 0
        return H

    ex = concurrent.futures.ThreadPoolExecutor(max_workers=_workers())
    futs = [ex.submit(oracle_hist, i) for i in range(R)]  # the oracle works while the device does

    # device pools: for every (distribution, width) and class c the pool shifted into [0, 2^c), as the benchmark stages them
    pools = {}
    for (d, w), base in pools_host.items():
        top = 24 if w == 4 else 16
        bt = torch.from_numpy(base.view(np.int32 if w == 4 else np.int16)).cuda()
        bt = _unsigned(bt)
        for c in range(8, top + 1):
            pools[(d, w, c)] = (bt >> (top - c)).to(torch.int32 if w == 4 else torch.int16)
    reqs = []
    for i in range(R):
        pool = pools[(str(tr["dist"][i]), int(tr["width"][i]), int(tr["cls"][i]))]
        o, n = int(tr["start"][i]), int(tr["n"][i])
        reqs.append((pool[o:o + n], int(tr["U"][i]), str(tr["kind"][i])))

    srv = ds.Server(hbm_budget_bytes=64 << 30, max_slots=64)
    tickets = [srv.submit(k, U, kind) for k, U, kind in reqs]  # all at once: admitted as slots and space free up
    errors = []
    overlapped = 0
    last_done = 0
    for i, (t, (k, U, kind)) in enumerate(zip(tickets, reqs)):
        res = srv.wait(t, timeout_s=120.0)
        if res["status"] != ds.OK:
            errors.append(f"request {i}: status {res['status']}")
            srv.release(t)
            continue
        if res["admit_ns"] < last_done:
            overlapped += 1  # admitted while an earlier request was still on the device
        last_done = max(last_done, res["done_ns"])
        H_ref = futs[i].result()
        H_dev = res["H"].cpu().numpy().view(np.uint32)
        if not np.array_equal(H_dev, H_ref):
            errors.append(f"request {i} (n={k.numel()} U={U} {kind}): histogram differs from the oracle")
        if kind == "sort":
            out = _unsigned(res["out"])
            sorted_ok = bool(torch.all(out[1:] >= out[:-1]).item()) if out.numel() > 1 else True
            counts = torch.bincount(out.to(torch.int64), minlength=U).to(torch.int32).cpu().numpy().view(np.uint32)
            if not (sorted_ok and counts.size == U and np.array_equal(counts, H_ref)):
                errors.append(f"request {i} (n={k.numel()} U={U}): sorted output is not the oracle's projection")
            alone = ds.sort(k, U)  # the same request alone
            if not torch.equal(alone, res["out"]):
                errors.append(f"request {i}: result in the mix differs from the request run alone")
        else:
            alone = ds.histogram(k, U)
            if not torch.equal(alone, res["H"]):
                errors.append(f"request {i}: histogram in the mix differs from the request run alone")
        srv.release(t)
    srv.close()
    ex.shutdown()
    assert ds.stream_status() == ds.OK
    assert not errors, errors[:5]
    assert overlapped > R // 4, f"only {overlapped} of {R} requests overlapped an earlier one on the device"
    kinds = set(tr["kind"][:R]) | set()
    assert {"sort", "histogram"} <= kinds and {2, 4} <= set(int(w) for w in tr["width"][:R])
    assert int(tr["U"][:R].max()) > (1 << 23)
