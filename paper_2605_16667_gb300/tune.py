"""Measure step 1's launch choices on this device and write the autotuner's table.

    python -m paper_2605_16667_gb300.tune [--out FILE] [--quick]

For every grid shape (log2 n, log2 U, key width) and skew class the script
times candidate launch choices of the histogram (Eq. (1)) on synthetic keys
of that class, with CUDA events on the launching stream, and writes one table
line per shape and class (the format dialsort_tune_table_load reads):

    log2n log2U key_bytes skew regime crn replicas threads blocks_per_sm

Skew classes and their inputs: 1 low conflict (uniform keys), 2 hot (Zipf
s = 1.1 over [0, U)), 3 runs (the uniform keys sorted); class 0 (unknown)
takes the candidate whose worst ratio to the cost model's time over the three
classes is smallest, and only if it beats the cost model on every class (so an
unprobed call is never slower than the cost model on any of them).  The cost model itself is always a candidate; a measured choice
replaces it only when it is faster by more than `margin` (3 %), and where it
is not the line says so with regime 0 (the cost model at that shape), so that
the table never overrides the cost model on a noise win.

Candidates: for each regime that fits the shape (32-bit and packed 16-bit
shared-memory sub-histograms with 1..32 copies, L2 atomics with and without
the warp CRN, the two-level regime where it applies) the CRN choice and the
copies are searched first with 1024-thread CTAs and the planner's grid; the
best of those is then tried with 256 / 512 / 1024 threads and 1, 2 or 4 CTAs
per SM.  Each candidate runs `reps` times after one warm-up launch and the
median counts; the keys (4n bytes, up to 512 MB) are larger than L2 at the
shapes that matter.
"""
from __future__ import annotations

import argparse
import math
import os
import sys
import time

import torch

import paper_2605_16667_gb300 as ds

DEFAULT_OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_table.txt")
SMEM_CAP = 227 * 1024


def keys_for(n: int, U: int, width: int, skew: int, seed: int = 20260321) -> torch.Tensor:
    """Synthetic keys of one skew class on the current device (int32 / int16 storage)."""
    g = torch.Generator(device="cuda")
    g.manual_seed(seed + 7919 * skew + U)
    if skew == 2:  # Zipf s = 1.1 over [0, U): inverse of the CDF of (k + 1)^-s
        w = torch.arange(1, U + 1, dtype=torch.float64, device="cuda").pow_(-1.1)
        cdf = torch.cumsum(w, 0)
        cdf /= cdf[-1].clone()
        u = torch.rand(n, generator=g, dtype=torch.float64, device="cuda")
        k = torch.searchsorted(cdf, u).clamp_(max=U - 1)
        del w, cdf, u
    else:
        k = torch.randint(0, U, (n,), generator=g, device="cuda", dtype=torch.int64)
        if skew == 3:
            k = torch.sort(k).values
    k = k.to(torch.int32)
    if width == 2:
        k = (k - (k >= 32768).to(torch.int32) * 65536).to(torch.int16)
    return k


def candidates_a(n: int, U: int, width: int):
    """Stage A: regime x CRN x copies, 1024 threads, the planner's grid."""
    out = []
    u32 = (U + 3) // 4 * 4 * 4
    u16 = ((U + 1) // 2 + 3) // 4 * 4 * 4
    for regime, copy in (("smem32", u32), ("smem16", u16)):
        if copy > SMEM_CAP:
            continue
        rep = 1
        while rep <= 32 and copy * rep <= SMEM_CAP:
            for crn in (2, 3, 1):
                out.append({"regime": regime, "crn": crn, "replicas": rep, "threads": 1024})
            rep *= 2
    for crn in (3, 1):
        out.append({"regime": "global_crn", "crn": crn, "threads": 1024})
    out.append({"regime": "global", "crn": 2, "threads": 1024})
    if width == 4 and n >= (1 << 20) and (1 << 16) < U <= (1 << 21):
        out.append({"regime": "two_level"})
    return out


def candidates_b(best: dict, sms: int):
    """Stage B: the best stage-A choice with other CTA sizes and grids."""
    if best.get("regime") in (None, "two_level"):
        return []
    out = []
    for threads in (256, 512, 1024):
        for per_sm in (0, 1, 2, 4):
            if per_sm * threads > 2048:
                continue
            c = dict(best, threads=threads)
            if per_sm:
                c["blocks"] = per_sm * sms
            if c != best:
                out.append(c)
    return out


def time_config(keys: torch.Tensor, U: int, config: dict | None, skew: int, reps: int) -> float:
    """Median ms of one histogram launch (with a workspace, as ds.histogram runs it)."""
    H = torch.empty(U, dtype=torch.int32, device="cuda")
    ws = torch.empty(max(ds.histogram_workspace_size(keys.numel(), U, keys.element_size()), 256),
                     dtype=torch.uint8, device="cuda")
    cfg = dict(config or {})
    cfg["skew"] = skew
    stream = torch.cuda.current_stream()
    ds.histogram(keys, U, H, config=cfg, ws=ws, stream=stream)  # warm-up
    times = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ds.histogram(keys, U, H, config=cfg, ws=ws, stream=stream)
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    if ds.stream_status() != ds.OK:
        raise RuntimeError(f"histogram reported an error for config {config}")
    times.sort()
    return times[len(times) // 2]


def valid(n: int, U: int, width: int, config: dict) -> bool:
    try:
        ds.plan_histogram(n, U, width, 0, **config)
        return True
    except ds.DialSortError:
        return False


def table_line(lg_n: int, lg_u: int, width: int, skew: int, c: dict | None, sms: int) -> str:
    if c is None:  # the cost model at this shape
        return f"{lg_n} {lg_u} {width} {skew} 0 0 0 0 0"
    regime = ds.REGIMES[c["regime"]]
    per_sm = c.get("blocks", 0) // sms if c.get("blocks") else 0
    return f"{lg_n} {lg_u} {width} {skew} {regime} {c.get('crn', 0)} {c.get('replicas', 0)} " \
           f"{c.get('threads', 0)} {per_sm}"


def tune_shape(lg_n: int, lg_u: int, width: int, sms: int, reps: int, margin: float, log) -> list[str]:
    n, U = 1 << lg_n, 1 << lg_u
    results = {}  # skew -> {key(config): ms}
    configs = {}
    for skew in (1, 2, 3):
        keys = keys_for(n, U, width, skew)
        res = {"model": time_config(keys, U, None, skew, reps)}
        configs["model"] = None
        best_key, best_t = "model", res["model"]
        for c in candidates_a(n, U, width):
            if not valid(n, U, width, c):
                continue
            k = repr(sorted(c.items()))
            res[k] = time_config(keys, U, c, skew, reps)
            configs[k] = c
            if res[k] < best_t:
                best_key, best_t = k, res[k]
        for c in candidates_b(configs[best_key] or {}, sms):
            if not valid(n, U, width, c):
                continue
            k = repr(sorted(c.items()))
            res[k] = time_config(keys, U, c, skew, reps)
            configs[k] = c
        results[skew] = res
        del keys
    lines = []
    for skew in (1, 2, 3):
        res = results[skew]
        k = min(res, key=res.get)
        chosen = configs[k] if res[k] * (1.0 + margin) < res["model"] else None
        log(f"  n=2^{lg_n} U=2^{lg_u} w={width} skew={skew}: model {res['model']:.4f} ms, best {res[k]:.4f} ms "
            f"{configs[k] if k != 'model' else 'model'} -> {'table' if chosen else 'model'}")
        lines.append(table_line(lg_n, lg_u, width, skew, chosen, sms))
    # unknown skew: a choice faster than the cost model on every class (by its worst ratio to the cost
    # model's time), among configs timed in every class; else the cost model
    common = set(results[1]) & set(results[2]) & set(results[3])

    def worst(k):
        return max(results[s][k] / results[s]["model"] for s in (1, 2, 3))

    k = min(common, key=worst)
    chosen = configs[k] if worst(k) * (1.0 + margin) < 1.0 else None
    lines.append(table_line(lg_n, lg_u, width, 0, chosen, sms))
    return lines


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--quick", action="store_true", help="a coarse grid (for a test run)")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--margin", type=float, default=0.03)
    args = ap.parse_args(argv)
    if not torch.cuda.is_available():
        sys.exit("the tuner measures on a CUDA device; none is visible")
    ds.tune_table_load(None)  # measure the cost model itself, not an older table
    sms = ds.lib().dialsort_device_sm_count()
    grid = []
    lg_ns = (20, 24) if args.quick else (16, 20, 24, 27)
    for lg_n in lg_ns:
        lg_us = (8, 16, 20, 24) if args.quick else (8, 10, 12, 14, 16, 18, 20, 22, 24, 26)
        for lg_u in lg_us:
            if lg_u <= lg_n + 2:
                grid.append((lg_n, lg_u, 4))
        for lg_u in ((8, 16) if args.quick else (8, 10, 12, 14, 16)):
            grid.append((lg_n, lg_u, 2))
    t0 = time.time()
    lines = [f"# step-1 launch choices measured on {torch.cuda.get_device_name()} ({sms} SMs), "
             f"median of {args.reps} launches; columns: log2n log2U key_bytes skew regime crn replicas threads "
             "blocks_per_sm (regime 0: the cost model)"]
    for lg_n, lg_u, width in grid:
        lines += tune_shape(lg_n, lg_u, width, sms, args.reps, args.margin, print)
        torch.cuda.empty_cache()
    with open(args.out, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(f"wrote {len(lines) - 1} entries to {args.out} in {time.time() - t0:.0f} s")
    ds.tune_table_load(args.out)


if __name__ == "__main__":
    main()
