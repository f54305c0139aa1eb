"""The reference arm of bench.py: the CPU oracle timed on the host on the benchmark's workload, printed
as the same JSON line with "impl": "reference".  Runs without a GPU (it never imports torch)."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BENCH = os.path.join(ROOT, "bench.py")


def _run(env_extra, *args):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, BENCH, "--impl", "reference", *args], capture_output=True, text=True,
                          env=env, cwd=ROOT, timeout=300)


def test_reference_arm_prints_one_line_of_the_contract():
    sys.path.insert(0, ROOT)
    import bench

    r = _run({"RANK": "0", "WORLD_SIZE": "1"}, "--steps", "3", "--warmup", "1", "--reference-seconds", "1")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "keys/s" and d["higher_is_better"] is True
    assert d["steps"] == 3 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["config"]["workload"] == bench.WORKLOAD
    n_s = d["config"]["sample_keys_per_step"]
    assert 1 << 16 <= n_s <= bench.N_KEYS
    assert d["value"] > 0 and abs(d["value"] - n_s * 3 / (d["ms_per_step"] * 3 / 1e3)) < 1e-6 * d["value"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"}, "--steps", "3", "--warmup", "1", "--reference-seconds", "1")
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
