#!/usr/bin/env python3
"""DialSort hot-path benchmark: histogram ingestion (Eq. 1) + ordered projection (Eq. 2).

Workload (one step): n = 2^28 uint32 keys drawn uniform on [0, 2^20) from the seeded
generator, sorted by one dialsort_sort call (zero H, ingest, offset scan, expand).
Keys stay resident in HBM; 1 GiB of keys and 1 GiB of output are larger than the
129 MB L2, so no flush is needed between steps.

Prints ONE JSON line (rank 0).  `value` is whole-job keys/s (all ranks; each GPU
runs an independent replica, so scaling is weak).  `e2e` repeats the measurement
through the same public C ABI with host (pinned) buffers, host->device and
device->host copies inside the timed region.  `roofline` is the dominant kernel's
algorithmic bytes per launch over its CUDA-event duration against the measured
HBM copy bandwidth.  `cpu_baseline` times the CPU oracle on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "keys/s & % of HBM roofline (hist+reconstruct); served p50/p99 latency"
N_KEYS = 1 << 28
UNIVERSE = 1 << 20
DIST = "uniform"
SEED_STREAM = 2 * 16 + 1
WORKLOAD = "dialsort_sort n=2^28 uint32 keys uniform on [0,2^20), histogram + reconstruction"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--e2e-steps", type=int, default=10)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-forms", action="store_true", help="skip the batched and served forms")
    p.add_argument("--served-seconds", type=float, default=10.0)
    p.add_argument("--reference-seconds", type=float, default=60.0,
                   help="host time the reference arm (the oracle) spends on its timed and warm-up steps")
    p.add_argument("--form", default="all",
                   choices=["all", "batched", "served", "radix", "paper", "autotune", "chunked"],
                   help="print only one form's measurement (batched, served, radix, the paper's workload grid, "
                        "or the autotuner against the cost model)")
    # workload-size overrides, for profiling smaller cases of the same kernels
    p.add_argument("--n", type=int, default=N_KEYS)
    p.add_argument("--U", type=int, default=UNIVERSE)
    p.add_argument("--dist", default=DIST)
    p.add_argument("--param", type=float, default=None, help="Zipf exponent (default 1.2)")
    p.add_argument("--width", type=int, default=4, choices=[2, 4], help="key width in bytes")
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2605_16667_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(phase: str):
    """DRAM bytes of one launch of kernel `phase` at the benchmark size, from the committed ncu summary
    (profiles/traffic.json), only if it was taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[phase]
        if e.get("source_hash") != kernel_source_hash():
            return None
        return e["bytes_per_launch_full"]
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples (every 10 ms) around the timed region.

    The sampler starts before the region and waits for its first line, so the region is covered from
    its start; `mark(True/False)` brackets the timed region, and `summary()` reports the samples taken
    inside it.  A short timed region (a few sorts of about a millisecond) still holds few samples, so
    the caller keeps the GPU busy with the same sort for a while after the region (`soak`), and those
    samples are reported beside the region's own ("soak_samples")."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, period_ms: int = 10):
        self.index = index
        self.period_ms = period_ms
        self.proc = None
        self.lines = []  # (time, line)
        self.window = [None, None]
        self.soak = [None, None]

    def _reader(self):
        import time
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line))

    def __enter__(self):
        import threading
        import time
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._reader, daemon=True).start()
            t0 = time.monotonic()
            while not self.lines and time.monotonic() - t0 < 3.0:  # sampling must be live before the region
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def mark(self, which: str, start: bool):
        import time
        (self.window if which == "region" else self.soak)[0 if start else 1] = time.monotonic()

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    @staticmethod
    def _parse(lines):
        sm, mx, reasons = [], None, set()
        for _, line in lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return sm, mx, reasons

    def summary(self):
        def within(w):
            if w[0] is None:
                return []
            end = w[1] if w[1] is not None else float("inf")
            return [(t, l) for t, l in self.lines if w[0] <= t <= end]
        sm, mx, reasons = self._parse(within(self.window))
        ssm, smx, sreasons = self._parse(within(self.soak))
        allsm = sm + ssm
        return {"sm_mhz": float(np.median(allsm)) if allsm else None, "sm_max_mhz": mx or smx,
                "reasons": sorted(reasons | sreasons), "samples": len(sm), "soak_samples": len(ssm),
                "period_ms": self.period_ms}


def cpu_baseline(n_sample: int, runs_budget_s: float = 15.0):
    """The CPU oracle (single thread) sorting a bounded sample of the same workload."""
    import gen
    import oracle

    keys = gen.keys(n_sample, UNIVERSE, DIST, stream=SEED_STREAM)
    oracle.sort(keys, UNIVERSE)  # warm-up
    times = []
    t_end = time.perf_counter() + runs_budget_s
    while time.perf_counter() < t_end or len(times) < 3:
        t0 = time.perf_counter()
        oracle.sort(keys, UNIVERSE)
        times.append(time.perf_counter() - t0)
        if len(times) >= 7:
            break
    best = min(times)
    return {"value": n_sample / best, "unit": "keys/s", "cores": 1, "kind": "oracle",
            "sample": f"n={n_sample} keys of the same distribution (uniform on [0,2^20)), oracle histogram + "
                      f"projection, best of {len(times)} runs"}, times


def job_throughput(ms_local: float, keys_per_rank: int, steps: int, dist=None, device=None):
    """Whole-job keys/s over the ranks: every rank sorted keys_per_rank keys per step; the job took as
    long as its slowest rank (max over ranks of the timed region).  Returns (keys/s, max ms)."""
    import torch

    ms = ms_local
    world = 1
    if dist is not None and dist.is_initialized():
        world = dist.get_world_size()
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return world * keys_per_rank * steps / (ms / 1e3), ms


def cpu_context(n_sample: int):
    """Context lines on the host cores, on the same sample as the oracle baseline: the multi-threaded CPU
    DialSort (per-thread histograms, bin-range expansion) on every core, and numpy's library sort."""
    import gen
    import cpu_baseline

    keys = gen.keys(n_sample, UNIVERSE, DIST, stream=SEED_STREAM)
    out = np.empty(n_sample, dtype=np.uint32)
    cores = cpu_baseline.threads()

    def best(fn, runs=5):
        fn()
        t = []
        for _ in range(runs):
            t0 = time.perf_counter()
            fn()
            t.append(time.perf_counter() - t0)
        return n_sample / min(t)

    par = best(lambda: cpu_baseline.sort(keys, UNIVERSE, out, cores))
    lib = best(lambda: np.sort(keys), runs=3)
    return {"parallel_cpu_dialsort": {"value": par, "unit": "keys/s", "cores": cores,
                                      "how": "count into per-thread histograms, sum, expand bin ranges (OpenMP)"},
            "library_sort": {"value": lib, "unit": "keys/s", "cores": 1, "how": "numpy.sort of the same keys"},
            "sample": f"n={n_sample} keys uniform on [0,2^20)"}


def _align(x, a):
    return (x + a - 1) // a * a


def run_radix(ds, torch, stream, n: int = 1 << 28, steps: int = 20):
    """DialSort-Radix on n full-range int32 keys: four base-256 passes plus the first digit's count.

    Algorithmic bytes: the count reads 4n; each pass reads and writes 4n (36n in all).
    """
    import gen

    peak, peak_kind = peaks()
    keys = torch.from_numpy(gen.words(n, stream=9 * 16 + 1).astype(np.uint32).view(np.int32)).cuda()
    out = torch.empty_like(keys)
    ws = torch.empty(ds.lib().dialsort_radix_workspace_size(n), dtype=torch.uint8, device="cuda")
    for _ in range(3):
        ds.radix_sort(keys, out=out, ws=ws, stream=stream)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        ds.radix_sort(keys, out=out, ws=ws, stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    ok = matches_library_sort(torch, keys, out) and ds.stream_status() == ds.OK
    gbs = 36 * n / (ms / 1e3) / 1e9
    return {"workload": f"dialsort_radix_sort_i32 n={n} full-range int32 (uniform 32-bit words)",
            "value": n / (ms / 1e3), "unit": "keys/s", "ms_per_sort": ms, "sorted_ok": ok,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "peak_source": peak_kind, "algorithmic_bytes_per_sort": 36 * n},
            "gpu_launches_per_sort": 5}


def matches_library_sort(torch, keys, out) -> bool:
    """The output is the input's multiset in order: equal, element by element, to torch's own sort of the
    input (a check outside every timed region; int32 order equals uint32 order for keys below 2^31, and
    16-bit keys are compared as unsigned values)."""
    if keys.dtype == torch.int16:
        keys, out = keys.to(torch.int32) & 0xFFFF, out.to(torch.int32) & 0xFFFF
    return bool(torch.equal(torch.sort(keys.flatten()).values, out.flatten()))


PAPER_NS = (10 ** 4, 10 ** 5, 10 ** 6, 10 ** 7)
PAPER_US = (256, 1024, 65536)
PAPER_DISTS = ("uniform", "paper_skew", "sorted", "reverse")


def run_paper(ds, torch, stream, runs: int = 7, warm: int = 3):
    """The paper's own workload grid (Sec. "Methodology"): N in {1e4, 1e5, 1e6, 1e7} x U in {256, 1024,
    65536} x {uniform, skewed (80 % of keys in [0, 0.05 U]), sorted, reverse}, each sorted by dialsort_sort
    `runs` times after `warm` warm-ups (the paper's best-of-7 protocol, with mean and CV), plus
    DialSort-Radix on 1e7 full-range int32 keys.  Inputs of these sizes stay in L2, and the small ones
    are bound by launch latency, so these are context lines beside the paper's CPU figures, not roofline
    figures."""
    import gen

    def timed(fn):
        for _ in range(warm):
            fn()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(runs + 1)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        for i in range(runs):
            fn()
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
        return np.array([ev[i].elapsed_time(ev[i + 1]) for i in range(runs)])

    rows = []
    sid = 12 * 16
    for N in PAPER_NS:
        for U in PAPER_US:
            for dist in PAPER_DISTS:
                sid += 1
                keys = torch.from_numpy(gen.keys(N, U, dist, stream=sid).view(np.int32)).cuda()
                out = torch.empty_like(keys)
                ws = torch.empty(ds.sort_workspace_size(N, U), dtype=torch.uint8, device="cuda")
                t = timed(lambda: ds.sort(keys, U, out=out, ws=ws, stream=stream))
                ok = matches_library_sort(torch, keys, out)
                rows.append({"N": N, "U": U, "dist": dist, "best_ms": float(t.min()), "mean_ms": float(t.mean()),
                             "cv": float(t.std() / t.mean()), "keys_per_s_best": N / (float(t.min()) / 1e3),
                             "sorted_ok": ok})
    n_rx = 10 ** 7
    words = torch.from_numpy(gen.words(n_rx, stream=sid + 1).astype(np.uint32).view(np.int32)).cuda()
    rx_out = torch.empty_like(words)
    rx_ws = torch.empty(ds.lib().dialsort_radix_workspace_size(n_rx), dtype=torch.uint8, device="cuda")
    t = timed(lambda: ds.radix_sort(words, out=rx_out, ws=rx_ws, stream=stream))
    radix = {"N": n_rx, "best_ms": float(t.min()), "mean_ms": float(t.mean()), "cv": float(t.std() / t.mean()),
             "keys_per_s_best": n_rx / (float(t.min()) / 1e3),
             "sorted_ok": matches_library_sort(torch, words, rx_out)}
    return {"workload": "the paper's grid: dialsort_sort of N uint32 keys, N in {1e4,1e5,1e6,1e7}, U in "
                        "{256,1024,65536}, uniform / skewed / sorted / reverse; DialSort-Radix on 1e7 int32",
            "protocol": f"{warm} warm-ups, best / mean / CV of {runs} runs (CUDA events per run)",
            "l2": "inputs smaller than L2 (context, not roofline)", "rows": rows, "radix": radix,
            "status": ds.stream_status()}


def run_autotune(ds, torch, stream, n: int = 1 << 27, reps: int = 7):
    """The universe sweep (n = 2^27 keys; U in {2^8, 2^12, 2^16, 2^20, 2^24, 2^26}, uniform and Zipf s = 1.1,
    plus 16-bit keys with U = 2^16): step 1 as the cost model plans it with no skew information (the
    planner without a table) against the measured table's plan for the probed skew class."""
    import os

    from paper_2605_16667_gb300 import tune

    if not os.path.exists(ds.TUNE_TABLE):
        return {"unavailable": "no measured tuning table next to the library"}
    cases = [(U, 4, d) for U in (1 << 8, 1 << 12, 1 << 16, 1 << 20, 1 << 24, 1 << 26) for d in ("uniform", "zipf")]
    cases += [(1 << 16, 2, "uniform"), (1 << 16, 2, "zipf")]

    def med(keys, U, skew):
        H = torch.empty(U, dtype=torch.int32, device="cuda")
        ws = torch.empty(max(ds.histogram_workspace_size(n, U, keys.element_size()), 256), dtype=torch.uint8,
                         device="cuda")
        for _ in range(2):
            ds.histogram(keys, U, H, ws=ws, skew=skew, stream=stream)
        t = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ds.histogram(keys, U, H, ws=ws, skew=skew, stream=stream)
            b.record(stream)
            b.synchronize()
            t.append(a.elapsed_time(b))
        t.sort()
        return t[len(t) // 2], H

    rows = []
    for U, w, d in cases:
        keys = tune.keys_for(n, U, w, 2 if d == "zipf" else 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        probe = ds.probe_skew(keys, U, stream)
        probe_ms = (time.perf_counter() - t0) * 1e3
        ds.tune_table_load(None)
        model_plan = ds.plan_histogram(n, U, w, 0)
        t_model, H_model = med(keys, U, None)
        ds.tune_table_load(ds.TUNE_TABLE)
        tuned_plan = ds.plan_histogram(n, U, w, probe["skew_class"])
        t_tuned, H_tuned = med(keys, U, probe["skew_class"])
        same = bool(torch.equal(H_model, H_tuned)) and int(H_tuned.to(torch.int64).sum().item()) == n
        keep = ("regime_name", "crn", "replicas", "threads", "blocks")
        rows.append({"U": U, "key_bytes": w, "distribution": "Zipf s=1.1" if d == "zipf" else "uniform",
                     "probe": {k: probe[k] for k in ("skew_name", "samples", "equal_neighbours",
                                                      "top_multiplicity")}, "probe_ms_host": round(probe_ms, 4),
                     "cost_model": {"plan": {k: model_plan[k] for k in keep}, "ms": t_model},
                     "tuned": {"plan": {k: tuned_plan[k] for k in keep}, "ms": t_tuned},
                     "speedup": t_model / t_tuned, "same_histogram": same})
        del keys, H_model, H_tuned
        torch.cuda.empty_cache()
    status = ds.stream_status()
    return {"workload": f"the universe sweep: histogram (Eq. (1)) of n = 2^27 keys, median of {reps} launches "
                        "after 2 warm-ups, keys larger than L2", "table_entries": ds.tune_table_size(),
            "rows": rows, "tuned_never_slower": all(r["tuned"]["ms"] <= r["cost_model"]["ms"] * 1.02 for r in rows),
            "tolerance": "2 % (launch-to-launch noise)", "all_same_histogram": all(r["same_histogram"] for r in rows),
            "status": status}


def run_chunked(ds, torch, stream, n: int = 1 << 28, U: int = 1 << 20, reps: int = 5):
    """Host-resident keys sorted two ways: serial (one copy of all keys to the device, then the sort) and
    chunked (dialsort_sort_chunked: each chunk's copy overlaps the ingestion of the chunk before; the
    projection runs once at the end).  Same keys, same output buffer on the device, events on `stream`."""
    import gen

    host = gen.keys(n, U, "uniform", stream=SEED_STREAM)
    pin = torch.from_numpy(host.view(np.int32)).pin_memory()
    del host
    d_keys = torch.empty(n, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    ws = torch.empty(ds.sort_workspace_size(n, U), dtype=torch.uint8, device="cuda")
    cs = torch.cuda.Stream()
    cws = {}

    def timed(fn):
        fn()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        ts.sort()
        return ts[len(ts) // 2]

    def copy_only():
        with torch.cuda.stream(stream):
            d_keys.copy_(pin, non_blocking=True)

    def sort_only():
        ds.sort(d_keys, U, out=out, ws=ws, stream=stream)

    def serial():
        copy_only()
        sort_only()

    t_copy, t_sort, t_serial = timed(copy_only), timed(sort_only), timed(serial)
    ref = out.clone()
    rows = []
    for chunk in (1 << 22, 1 << 24, 1 << 26):
        need = ds.lib().dialsort_chunked_workspace_size(n, U, 4, chunk, 1)
        cws[chunk] = torch.empty(need, dtype=torch.uint8, device="cuda")
        out.fill_(-1)
        t = timed(lambda: ds.sort_chunked(pin, U, out, chunk_keys=chunk, ws=cws[chunk], stream=stream,
                                          copy_stream=cs))
        rows.append({"chunk_keys": chunk, "ms": t, "keys_per_s": n / (t / 1e3), "same_output": bool(torch.equal(out, ref))})
        del cws[chunk]
    best = min(rows, key=lambda r: r["ms"])
    status = ds.stream_status()
    return {"workload": f"dialsort_sort of n = 2^28 uint32 keys, U = 2^20, uniform, in page-locked host memory "
                        f"(1 GiB), output on the device; median of {reps}",
            "copy_ms": t_copy, "device_sort_ms": t_sort, "serial_ms": t_serial,
            "serial_keys_per_s": n / (t_serial / 1e3), "chunked": rows, "best_chunked_ms": best["ms"],
            "saved_ms": t_serial - best["ms"], "lower_bound_ms": max(t_copy, t_sort),
            "how": "serial: one cudaMemcpyAsync of all keys, then dialsort_sort; chunked: dialsort_sort_chunked with "
                   "two staging buffers, copies on a second stream", "status": status}


def run_batched(ds, torch, stream, reps: int = 3):
    """4096 independent instances in one persistent launch vs per-request plain launches.

    n_i log-uniform in [2^10, 2^22], U_i log-uniform in [2^8, 2^20], each instance's distribution
    drawn uniformly from {uniform, Zipf s=1.2, all equal}; uint32 keys; histogram + projection.
    """
    import concurrent.futures

    import gen

    count = 4096
    ns, us, dists = gen.batch_workload(count)
    koff = np.zeros(count + 1, dtype=np.int64)
    hoff = np.zeros(count + 1, dtype=np.int64)
    for i in range(count):
        koff[i + 1] = koff[i] + _align(int(ns[i]), 64)
        hoff[i + 1] = hoff[i] + _align(int(us[i]), 64)
    host = np.empty(int(koff[-1]), dtype=np.uint32)

    def fill(i):
        gen.batch_keys(i, ns[i], us[i], dists[i], out=host[koff[i]:koff[i] + ns[i]])

    with concurrent.futures.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        list(ex.map(fill, range(count)))
    keys_d = torch.from_numpy(host.view(np.int32)).cuda()
    out_d = torch.empty_like(keys_d)
    H_d = torch.empty(int(hoff[-1]), dtype=torch.int32, device="cuda")
    kv = [keys_d[koff[i]:koff[i] + ns[i]] for i in range(count)]
    ov = [out_d[koff[i]:koff[i] + ns[i]] for i in range(count)]
    hv = [H_d[hoff[i]:hoff[i] + us[i]] for i in range(count)]
    total_keys = int(ns.sum())
    algo_bytes = int(8 * ns.sum() + 12 * us.sum())

    b = ds.Batch(kv, [int(u) for u in us], H=hv, out=ov, sort=True)
    b.launch(stream)
    torch.cuda.synchronize()
    ok = ds.stream_status() == ds.OK
    # every instance against the same instance through the single-instance entry points (outside any
    # timing; the full comparison with the CPU oracle is tests/test_gpu_fullsize.py)
    for i in range(count):
        ok = ok and torch.equal(hv[i], ds.histogram(kv[i], int(us[i]))) and torch.equal(ov[i], ds.sort(kv[i], int(us[i])))
    for i in (0, count // 2, count - 1):
        ok = ok and bool(np.array_equal(ov[i].cpu().numpy().view(np.uint32), np.sort(host[koff[i]:koff[i] + ns[i]])))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        b.launch(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    batched_ms = e0.elapsed_time(e1) / reps
    # the same launch captured in a CUDA graph
    g = torch.cuda.CUDAGraph()
    s2 = torch.cuda.Stream()
    with torch.cuda.stream(s2):
        with torch.cuda.graph(g, stream=s2):
            b.launch(s2)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        g.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    graph_ms = e0.elapsed_time(e1) / reps
    del g
    b.close()
    # per-request plain launches on one stream (C loop: all arrivals at t = 0)
    entries = [(kv[i], int(us[i]), "sort", 0) for i in range(count)]
    ds.replay(entries[:64], use_server=False, hbm_budget_bytes=8 << 30)  # warm-up
    _, plain_wall = ds.replay(entries, use_server=False, hbm_budget_bytes=8 << 30)
    plain_ms = plain_wall / 1e6
    best = min(batched_ms, graph_ms)
    return {"workload": "4096 instances, n_i log-uniform [2^10,2^22], U_i log-uniform [2^8,2^20], "
                        "uniform/Zipf 1.2/all-equal, uint32, histogram + projection",
            "total_keys": total_keys, "batched_ms": batched_ms, "graph_ms": graph_ms,
            "plain_launches_ms": plain_ms, "batched_keys_per_s": total_keys / (best / 1e3),
            "plain_keys_per_s": total_keys / (plain_ms / 1e3), "speedup_vs_plain": plain_ms / best,
            "hbm_frac": algo_bytes / (best / 1e3) / 1e9 / peaks()[0], "algorithmic_bytes": algo_bytes,
            "launches": 1, "checked": ok,
            "checked_how": "every instance's H and output equal to the instance run alone through "
                           "dialsort_histogram / dialsort_sort; three also equal to numpy's sort"}


def run_served(ds, torch, seconds: float = 10.0, warm: float = 1.0, rate: float = 2000.0):
    """Poisson request stream through the server vs per-request plain launches (same trace).

    n log-uniform [2^12,2^26], U log-uniform [2^8,2^24], uint32/uint16 keys 50/50 (uint16 => U <= 2^16),
    sort/histogram 50/50, uniform/Zipf 1.2 50/50, 64 GB HBM budget.  Keys are pre-staged on the device:
    for each (distribution, width) one base array of 2^26 keys drawn over the largest universe, and
    for each power of two 2^c the keys shifted right so they lie in [0, 2^c); a request with universe
    U reads a slice of the class floor(log2 U), so every key is < U.
    """
    import gen

    tr = gen.served_trace(rate, seconds, warm)
    count, arrivals, ns, us = len(tr["n"]), tr["arrivals"], tr["n"], tr["U"]
    pools = {}
    for d in ("uniform", "zipf"):
        for wd in (4, 2):
            base = gen.served_pool(d, wd)
            bt = torch.from_numpy(base.view(np.int32 if wd == 4 else np.int16)).cuda()
            if wd == 2:
                bt = bt.to(torch.int32) & 0xFFFF
            top = 24 if wd == 4 else 16
            for c in range(8, top + 1):
                pools[(d, wd, c)] = (bt >> (top - c)).to(torch.int32 if wd == 4 else torch.int16)
            del bt
    entries = []
    for i in range(count):
        pool = pools[(str(tr["dist"][i]), int(tr["width"][i]), int(tr["cls"][i]))]
        o = int(tr["start"][i])
        entries.append((pool[o:o + ns[i]], int(us[i]), str(tr["kind"][i]), int(arrivals[i] * 1e9)))
    meas = arrivals >= warm
    out = {"workload": f"Poisson {rate:.0f} req/s for {seconds:.0f} s after {warm:.0f} s warm-up "
                       f"({int(meas.sum())} measured requests), n log-uniform [2^12,2^26], U log-uniform "
                       "[2^8,2^24], uint32/uint16, sort/histogram, uniform/Zipf 1.2, 64 GB budget",
           "requests": int(meas.sum())}
    for name, use_server in (("served", True), ("plain_launches", False)):
        res, wall = ds.replay(entries, use_server=use_server, hbm_budget_bytes=64 << 30, max_slots=64)
        lat = (res["done_ns"].astype(np.float64) - res["arrival_ns"].astype(np.float64))[meas] / 1e6
        span = (res["done_ns"][meas].max() - res["arrival_ns"][meas].min()) / 1e9
        st_vals, st_counts = np.unique(res["status"], return_counts=True)
        out[name] = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                     "mean_ms": float(lat.mean()), "keys_per_s": float(ns[meas].sum() / span),
                     "all_ok": bool(np.all(res["status"] == 0)), "wall_s": wall / 1e9,
                     "status_counts": {int(v): int(c) for v, c in zip(st_vals, st_counts)}}
    # rate sweep: the trace's first 4000 requests with their arrival gaps scaled to 2k, 8k and 32k req/s, and
    # all at once (closed loop: the largest backlog), through the server and through plain launches
    sweep_n = min(4000, count)
    base_ns = np.array([e[3] for e in entries[:sweep_n]], dtype=np.float64)
    sweep = []
    for r in (2000.0, 8000.0, 32000.0, None):
        scale = 0.0 if r is None else rate / r
        ents = [(e[0], e[1], e[2], int(base_ns[i] * scale)) for i, e in enumerate(entries[:sweep_n])]
        row = {"rate_req_s": r if r is not None else "closed loop (all at t = 0)", "requests": sweep_n}
        for name, use_server in (("served", True), ("plain_launches", False)):
            res, wall = ds.replay(ents, use_server=use_server, hbm_budget_bytes=64 << 30, max_slots=64)
            lat = (res["done_ns"].astype(np.float64) - res["arrival_ns"].astype(np.float64)) / 1e6
            span = (res["done_ns"].max() - res["arrival_ns"].min()) / 1e9
            row[name] = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                         "keys_per_s": float(ns[:sweep_n].sum() / span), "all_ok": bool(np.all(res["status"] == 0))}
        sweep.append(row)
    out["rate_sweep"] = sweep
    # results, not just status: every 10th request of the trace through the server (all submitted at once,
    # so they overlap), each compared with the same request run alone (untimed)
    srv = ds.Server(hbm_budget_bytes=64 << 30, max_slots=64)
    sample = list(range(0, count, 10))
    tickets = [srv.submit(entries[i][0], entries[i][1], entries[i][2]) for i in sample]
    match = 0
    for i, t in zip(sample, tickets):
        keys_i, U_i, kind_i, _ = entries[i]
        res = srv.wait(t, timeout_s=120.0)
        if res["status"] == ds.OK:
            same = torch.equal(res["out"], ds.sort(keys_i, U_i)) if kind_i == "sort" else \
                torch.equal(res["H"], ds.histogram(keys_i, U_i))
            match += int(same)
        srv.release(t)
    srv.close()
    out["results_checked"] = {"requests": len(sample), "equal_to_alone": match,
                              "how": "every 10th request of the trace served together, each result compared with "
                                     "the same request run alone (the full comparison with the CPU oracle is "
                                     "tests/test_gpu_fullsize.py)"}
    for name in ("served", "plain_launches"):
        out[name]["all_ok"] = out[name]["all_ok"] and match == len(sample)
    del pools
    return out


def run_reference(args, rank, world):
    """The oracle on host cores, on this workload's config and metric (bounded sample per step)."""
    if rank != 0:
        return 0
    import gen
    import oracle

    # calibrate a per-step sample so that all steps finish in about --reference-seconds (a minute)
    cal = gen.keys(1 << 20, UNIVERSE, DIST, stream=SEED_STREAM)
    t0 = time.perf_counter()
    oracle.sort(cal, UNIVERSE)
    rate = (1 << 20) / max(time.perf_counter() - t0, 1e-6)
    per_step = args.reference_seconds / max(1, args.steps + args.warmup)
    n_s = int(min(N_KEYS, max(1 << 16, rate * per_step)))
    keys = gen.keys(n_s, UNIVERSE, DIST, stream=SEED_STREAM)
    for _ in range(args.warmup):
        oracle.sort(keys, UNIVERSE)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.sort(keys, UNIVERSE)
    dt = time.perf_counter() - t0
    value = n_s * args.steps / dt
    sample = f"n={n_s} keys per step (uniform on [0,2^20)), single-threaded oracle histogram + projection"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "keys/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_keys_per_step": n_s},
            "cpu_baseline": {"value": value, "unit": "keys/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "keys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch

    import gen
    import paper_2605_16667_gb300 as ds

    torch.cuda.set_device(local_rank)
    if args.form != "all":
        stream = torch.cuda.current_stream()
        if args.form == "batched":
            res = run_batched(ds, torch, stream)
        elif args.form == "radix":
            res = run_radix(ds, torch, stream, n=args.n)
        elif args.form == "paper":
            res = run_paper(ds, torch, stream)
        elif args.form == "autotune":
            res = run_autotune(ds, torch, stream)
        elif args.form == "chunked":
            res = run_chunked(ds, torch, stream)
        else:
            res = run_served(ds, torch, seconds=args.served_seconds)
        print(json.dumps({"form": args.form, **res}), flush=True)
        return 0
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if dist is not None:
            dist.barrier()

    n, U, w = args.n, args.U, args.width
    keys_host = gen.keys(n, U, args.dist, width=w, param=args.param, stream=SEED_STREAM + 1000 * rank)
    keys = torch.from_numpy(keys_host.view(np.int32 if w == 4 else np.int16)).cuda()
    out = torch.empty_like(keys)
    ws = torch.empty(ds.sort_workspace_size(n, U), dtype=torch.uint8, device="cuda")
    plan = ds.plan_histogram(n, U, w)
    sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
    # kernels of ours per sort: two-level: partition, split, schedule, counting fused with the projection;
    # otherwise the ingestion kernel and the (fused offsets + expansion) projection kernel
    launches_per_step = 4 if plan["regime_name"] == "two_level" else 2
    H = torch.empty(U, dtype=torch.int32, device="cuda")
    rws = torch.empty(ds.reconstruct_workspace_size(U, n), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        ds.sort(keys, U, out=out, ws=ws, stream=stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    if ds.stream_status() != ds.OK:
        raise RuntimeError("device error word set during warm-up")

    # ---- timed region: K sort steps, device-resident keys
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    e0, e1 = ev[0], ev[-1]
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        clk.mark("region", True)
        e0.record(stream)
        for i in range(args.steps):
            step()
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
        clk.mark("region", False)
        # the same sort for about 0.3 s more (untimed), so that the clock record holds enough samples
        clk.mark("soak", True)
        t_soak = time.monotonic()
        while time.monotonic() - t_soak < 0.3:
            for _ in range(16):
                step()
            torch.cuda.synchronize()
        clk.mark("soak", False)
    barrier()
    ms = e0.elapsed_time(e1)
    per_step = np.array([ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)])
    step_stats = {"best_ms": float(per_step.min()), "mean_ms": float(per_step.mean()),
                  "std_ms": float(per_step.std()), "cv": float(per_step.std() / per_step.mean())}
    value, ms = job_throughput(ms, n, args.steps, dist, torch.device("cuda", local_rank))

    # sanity on the last result (outside the timed region): the input's multiset in order, sum(H) = n
    sorted_ok = matches_library_sort(torch, keys, out)
    Hs = ws[: 4 * U].view(torch.int32)
    hist_sum_ok = int(Hs.to(torch.int64).sum().item()) == n
    status = ds.stream_status()

    # ---- per-phase CUDA-event timing on the same stream (for the roofline)
    def timed(fn, reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    reps = max(10, min(args.steps, 100))
    hist_ms = timed(lambda: ds.histogram(keys, U, H, stream=stream), reps)
    offs_ms = timed(lambda: ds.lib().dialsort_offsets(H.data_ptr(), U, n, rws.data_ptr(), rws.numel(),
                                                      stream.cuda_stream), reps)
    recon_ms = timed(lambda: ds.reconstruct(H, U, n, out, ws=rws, stream=stream), reps)
    expand_ms = max(recon_ms - offs_ms, 1e-9)
    peak, peak_kind = peaks()
    # the kernels inside the sort itself: CUDA events between its stages (the two-level form: pass 1,
    # split + schedule, counting fused with the projection, long runs), median of `reps` sorts
    st_runs = np.array([ds.sort_stage_times(keys, U, out, ws, stream=stream) for _ in range(reps)])
    stage_ms = [float(x) for x in np.median(st_runs, axis=0)]
    if len(stage_ms) == 4:
        stage_names = ["partition (pass 1)", "split + schedule", "count + projection (fused)", "long runs"]
        # algorithmic bytes: pass 1 reads the keys; the fused kernel zeroes/adds/reads H and writes the keys
        stage_bytes = [w * n, 0, w * n + 12 * U, 0]
        kernel_of = ["hier_partition_kernel", "hier_split_kernel + hier_sched_kernel", "hier_sort_kernel",
                     "hier_long_kernel"]
    else:
        stage_names, stage_bytes, kernel_of = ["sort"], [2 * w * n + 12 * U], ["sort kernels"]
    i_dom = int(np.argmax(stage_ms))
    dom_ms, dom_bytes = stage_ms[i_dom], stage_bytes[i_dom]
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": ncu_traffic(kernel_of[i_dom]), "kernel": f"{kernel_of[i_dom]} ({stage_names[i_dom]})",
                "peak_source": peak_kind, "algorithmic_bytes_per_launch": dom_bytes,
                "stages_ms": dict(zip(stage_names, stage_ms)),
                "how": "CUDA events between the sort's stages on its stream (dialsort_sort_stage_times), median "
                       f"of {reps} sorts after the timed region"}
    step_bytes = 2 * w * n + 12 * U
    whole = {"achieved_gbs": step_bytes / (ms / args.steps / 1e3) / 1e9}
    whole["frac_of_peak"] = whole["achieved_gbs"] / peak

    # ---- end to end through the public API with host buffers.  Zero-copy: dialsort_sort gets the pinned
    # host input and output themselves; its kernels read the keys and write the sorted keys across the
    # CPU-GPU link.  For context, the staged form (copy in, sort on the device, copy out) is timed too.
    pin_in = torch.empty(n, dtype=keys.dtype, pin_memory=True)
    pin_in.copy_(torch.from_numpy(keys_host.view(np.int32 if w == 4 else np.int16)))
    pin_out = torch.empty(n, dtype=keys.dtype, pin_memory=True)
    d_in = torch.empty_like(keys)

    def e2e_step():
        ds.sort(pin_in, U, out=pin_out, ws=ws, stream=stream)

    def staged_step():
        d_in.copy_(pin_in, non_blocking=True)
        ds.sort(d_in, U, out=out, ws=ws, stream=stream)
        pin_out.copy_(out, non_blocking=True)

    def time_e2e(fn, steps):
        for _ in range(2 if steps else 0):
            fn()
        torch.cuda.synchronize()
        barrier()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        t = max(e0.elapsed_time(e1), 1e-9)
        v, _ = job_throughput(t, n, steps, dist, torch.device("cuda", local_rank))
        return v if steps else None

    # Pipelined staged form: the same three operations per step, with consecutive steps overlapped on three
    # streams (step i + 1's copy in runs during step i's sort and copy out; the two directions of the link
    # carry data at the same time).  Inputs and outputs on the device are double-buffered.
    d_in2 = [d_in, torch.empty_like(keys)]
    d_out2 = [out, torch.empty_like(keys)]
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    def pipelined(steps):
        done_sort, done_out = [], []
        s_in.wait_stream(stream)
        for i in range(steps):
            j = i & 1
            if i >= 2:
                s_in.wait_event(done_sort[i - 2])  # the sort that read d_in2[j] has finished
            with torch.cuda.stream(s_in):
                d_in2[j].copy_(pin_in, non_blocking=True)
            stream.wait_stream(s_in)
            if i >= 2:
                stream.wait_event(done_out[i - 2])  # d_out2[j] has been copied out
            ds.sort(d_in2[j], U, out=d_out2[j], ws=ws, stream=stream)
            ev_s = torch.cuda.Event()
            ev_s.record(stream)
            done_sort.append(ev_s)
            s_out.wait_event(ev_s)
            with torch.cuda.stream(s_out):
                pin_out.copy_(d_out2[j], non_blocking=True)
            ev_o = torch.cuda.Event()
            ev_o.record(s_out)
            done_out.append(ev_o)
        stream.wait_stream(s_out)

    def time_pipelined(steps):
        if not steps:
            return None
        pipelined(2)
        torch.cuda.synchronize()
        barrier()
        e0.record(stream)
        pipelined(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        v, _ = job_throughput(max(e0.elapsed_time(e1), 1e-9), n, steps, dist, torch.device("cuda", local_rank))
        return v

    e2e_steps = min(args.e2e_steps, args.steps)
    e2e_value = time_e2e(e2e_step, e2e_steps)
    staged_value = time_e2e(staged_step, e2e_steps)
    pipe_value = time_pipelined(e2e_steps)
    head = pin_out.numpy()[: 1 << 20].view(np.uint32 if w == 4 else np.uint16)
    e2e_ok = bool(np.all(head[1:] >= head[:-1])) if e2e_steps else None
    staged = {"value": staged_value, "how": "pinned host keys copied in (cudaMemcpyAsync), dialsort_sort on the "
              "device, sorted keys copied out; copies inside the timed region"}
    zero_copy = {"value": e2e_value, "how": "dialsort_sort given the pinned host buffers themselves: its kernels "
                 "read and write host memory across the CPU-GPU link"}
    piped = {"value": pipe_value, "how": "copy in, dialsort_sort on the device, copy out, with consecutive steps "
             "overlapped on three streams (double-buffered device input and output); every step's copies inside "
             "the timed region"}
    ranked = sorted([zero_copy, staged, piped], key=lambda f: f["value"] or 0, reverse=True)
    best = ranked[0]
    e2e = {"value": best["value"], "unit": "keys/s",
           "h2d_bytes_per_step": w * n, "d2h_bytes_per_step": w * n, "steps": e2e_steps,
           "host_output_sorted": e2e_ok, "how": best["how"] + " (the fastest of three host-buffer forms)",
           "other_forms": ranked[1:]}

    cpu = None
    cpu_ctx = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu, _ = cpu_baseline(1 << 25)
        try:
            cpu_ctx = cpu_context(1 << 25)
        except Exception as exc:  # a context line only: never fails the benchmark
            cpu_ctx = {"unavailable": str(exc)[:200]}

    # the batched and served forms, each against per-request plain launches
    forms = {}
    if not args.no_forms and n == N_KEYS:
        del keys, out, ws, rws, pin_in, pin_out, d_in, d_in2, d_out2
        torch.cuda.empty_cache()
        forms["batched"] = run_batched(ds, torch, stream)
        torch.cuda.empty_cache()
        forms["served"] = run_served(ds, torch, seconds=args.served_seconds)
        torch.cuda.empty_cache()
        forms["radix"] = run_radix(ds, torch, stream)
        torch.cuda.empty_cache()
        try:  # context lines only: never fails the benchmark
            forms["paper_grid"] = run_paper(ds, torch, stream)
        except Exception as exc:
            forms["paper_grid"] = {"unavailable": str(exc)[:200]}
        torch.cuda.empty_cache()
        try:
            forms["autotune"] = run_autotune(ds, torch, stream)
        except Exception as exc:
            forms["autotune"] = {"unavailable": str(exc)[:200]}
        torch.cuda.empty_cache()
        forms["chunked_ingest"] = run_chunked(ds, torch, stream)
        torch.cuda.empty_cache()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "keys/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32" if w == 4 else "u16", "data": "synthetic",
            "config": {"workload": WORKLOAD if (n, U, args.dist) == (N_KEYS, UNIVERSE, DIST)
                       else f"dialsort_sort n={n} U={U} {args.dist}", "n": n, "U": U, "distribution": args.dist,
                       "key_bytes": w, "zipf_s": (args.param or 1.2) if "zipf" in args.dist else None,
                       "histogram_regime": plan["regime_name"],
                       "l2": f"inputs larger than L2 ({w * n / 2**30:.3g} GiB keys, same output), no flush"
                       if w * n > 129e6 else "inputs smaller than L2: numbers include L2 residency",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline, "whole_step_hbm": whole,
            "phases_ms": {"histogram": hist_ms, "offsets": offs_ms, "expand": expand_ms, "reconstruct": recon_ms},
            "cpu_baseline": cpu, "cpu_context": cpu_ctx, "e2e": e2e, "clocks": clk.summary(),
            "gpu_launches": launches_per_step * args.steps, "step_stats": step_stats,
            "keys_per_sm_clock": value / world / (sms * 1e6 * (clk.summary()["sm_mhz"] or 2070.0)), "status": status, "hist_sum_ok": hist_sum_ok, "sorted_ok": sorted_ok,
        }
        line.update(forms)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
