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
    # workload-size overrides, for profiling smaller cases of the same kernels
    p.add_argument("--n", type=int, default=N_KEYS)
    p.add_argument("--U", type=int, default=UNIVERSE)
    p.add_argument("--dist", default=DIST)
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


def ncu_traffic(kernel: str):
    """DRAM bytes per launch for `kernel` from the committed ncu summary, if it was taken on this source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[kernel]
        if e.get("source_hash") != kernel_source_hash():
            return None
        return e["bytes_per_launch_full"]
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        for line in (self.out or "").splitlines():
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
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


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


def run_reference(args, rank, world):
    """The oracle on host cores, on this workload's config and metric (bounded sample per step)."""
    if rank != 0:
        return 0
    import gen
    import oracle

    # calibrate a per-step sample so that all steps finish in about a minute
    cal = gen.keys(1 << 20, UNIVERSE, DIST, stream=SEED_STREAM)
    t0 = time.perf_counter()
    oracle.sort(cal, UNIVERSE)
    rate = (1 << 20) / max(time.perf_counter() - t0, 1e-6)
    per_step = 60.0 / max(1, args.steps + args.warmup)
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
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if dist is not None:
            dist.barrier()

    n, U = args.n, args.U
    keys_host = gen.keys(n, U, args.dist, stream=SEED_STREAM + 1000 * rank)
    keys = torch.from_numpy(keys_host.view(np.int32)).cuda()
    out = torch.empty_like(keys)
    ws = torch.empty(ds.sort_workspace_size(n, U), dtype=torch.uint8, device="cuda")
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
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * n * args.steps / (ms / 1e3)

    # sanity on the last result (outside the timed region): sorted, sum(H) = n
    sorted_ok = bool(torch.all(out[1:] >= out[:-1]).item())
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
    hist_bytes = 4 * n + 8 * U   # read keys, zero H, write H
    recon_bytes = 4 * n + 4 * U  # read H, write the keys
    if hist_ms >= recon_ms:
        dom, dom_bytes, dom_ms, kname = "histogram (zero H + ingest)", hist_bytes, hist_ms, "hist_kernel"
    else:
        dom, dom_bytes, dom_ms, kname = "reconstruct (offsets + expand)", recon_bytes, recon_ms, "expand_kernel"
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": ncu_traffic(kname), "kernel": dom, "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": dom_bytes}
    step_bytes = 8 * n + 12 * U
    whole = {"achieved_gbs": step_bytes / (ms / args.steps / 1e3) / 1e9}
    whole["frac_of_peak"] = whole["achieved_gbs"] / peak

    # ---- end to end through the public API with host buffers
    pin_in = torch.from_numpy(keys_host.view(np.int32)).pin_memory()
    pin_out = torch.empty(n, dtype=torch.int32).pin_memory()
    d_in = torch.empty_like(keys)

    def e2e_step():
        d_in.copy_(pin_in, non_blocking=True)
        ds.sort(d_in, U, out=out, ws=ws, stream=stream)
        pin_out.copy_(out, non_blocking=True)

    e2e_steps = min(args.e2e_steps, args.steps)
    for _ in range(2 if e2e_steps else 0):
        e2e_step()
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max(e0.elapsed_time(e1), 1e-9)
    if dist is not None:
        t = torch.tensor([e2e_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    head = pin_out.numpy()[: 1 << 20].view(np.uint32)
    e2e_ok = bool(np.all(head[1:] >= head[:-1])) if e2e_steps else None
    e2e = {"value": world * n * e2e_steps / (e2e_ms / 1e3) if e2e_steps else None, "unit": "keys/s",
           "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 4 * n, "steps": e2e_steps,
           "host_output_sorted": e2e_ok}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu, _ = cpu_baseline(1 << 25)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "keys/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD if (n, U, args.dist) == (N_KEYS, UNIVERSE, DIST)
                       else f"dialsort_sort n={n} U={U} {args.dist}", "n": n, "U": U, "distribution": args.dist,
                       "key_bytes": 4,
                       "l2": "inputs larger than L2 (1 GiB keys, 1 GiB output), no flush",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline, "whole_step_hbm": whole,
            "phases_ms": {"histogram": hist_ms, "offsets": offs_ms, "expand": expand_ms, "reconstruct": recon_ms},
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(),
            "gpu_launches": 3 * args.steps, "status": status, "hist_sum_ok": hist_sum_ok, "sorted_ok": sorted_ok,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
