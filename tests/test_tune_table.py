"""The autotuner's measured table: parsing, nearest-entry lookup, fallbacks (host only, no GPU)."""
import os
import subprocess
import sys

import pytest

from conftest import ROOT


@pytest.fixture
def ds():
    import __graft_entry__ as g

    g.build()
    import paper_2605_16667_gb300 as ds

    yield ds
    ds.tune_table_load(ds.TUNE_TABLE if os.path.exists(ds.TUNE_TABLE) else None)


TABLE = """# test table
20 8 4 2 1 1 8 512 2
20 8 4 1 1 2 1 1024 0
27 20 4 1 5 2 0 512 0
27 20 4 2 4 3 0 1024 1
24 12 2 3 2 1 1 256 0
27 16 4 0 0 0 0 0 0
27 24 4 2 1 1 1 1024 0
not a line
27 18 4 1 6 0 0 0 0
"""


def _write(tmp_path, text=TABLE):
    p = tmp_path / "t.txt"
    p.write_text(text)
    return str(p)


def test_load_counts_entries_and_rejects_missing_file(ds, tmp_path):
    path = _write(tmp_path)
    ds.tune_table_load(path)
    assert ds.tune_table_size() == 8  # comment and malformed lines skipped
    with pytest.raises(ds.DialSortError):
        ds.tune_table_load(str(tmp_path / "absent.txt"))
    assert ds.tune_table_size() == 8  # the old table stays
    ds.tune_table_load(None)
    assert ds.tune_table_size() == 0


def test_exact_and_nearest_entries(ds, tmp_path):
    ds.tune_table_load(_write(tmp_path))
    p = ds.plan_histogram(1 << 20, 1 << 8, 4, 2)  # exact: skew 2
    assert (p["regime_name"], p["crn"], p["replicas"], p["threads"]) == ("smem32", 1, 8, 512)
    assert p["blocks"] >= 1 and p["skew"] == 2
    p = ds.plan_histogram(1 << 20, 1 << 8, 4, 1)  # same shape, skew 1
    assert (p["regime_name"], p["crn"], p["replicas"], p["threads"]) == ("smem32", 2, 1, 1024)
    p = ds.plan_histogram(1 << 21, 300, 4, 1)  # nearest: log2 n 21, log2 U 8 -> distance 1
    assert (p["regime_name"], p["replicas"]) == ("smem32", 1)
    # 2^27 x 2^20, skew 1: the measured entry names the plain L2 regime with 512 threads, and it stands
    # (the two-level pass is taken only where an entry names it, or where there is no entry)
    p = ds.plan_histogram(1 << 27, 1 << 20, 4, 1)
    assert p["regime_name"] == "global" and p["threads"] == 512
    p = ds.plan_histogram(1 << 27, 1 << 18, 4, 1)  # an entry naming the two-level regime
    assert p["regime_name"] == "two_level"
    p = ds.plan_histogram(1 << 24, 1 << 12, 2, 3)  # 16-bit keys, runs
    assert (p["regime_name"], p["crn"], p["threads"]) == ("smem16", 1, 256)


def test_entries_that_do_not_apply_fall_back_to_the_cost_model(ds, tmp_path):
    ds.tune_table_load(None)
    model = {k: ds.plan_histogram(*k) for k in
             [(1 << 20, 1 << 8, 4, 3), (1 << 27, 1 << 24, 4, 2), (1 << 27, 1 << 16, 4, 0), (1 << 12, 1 << 26, 4, 2)]}
    ds.tune_table_load(_write(tmp_path))
    # no entry for skew 3 at width 4 near 2^20 x 2^8 (the 16-bit runs entry has another width)
    assert ds.plan_histogram(1 << 20, 1 << 8, 4, 3) == model[(1 << 20, 1 << 8, 4, 3)]
    # an entry naming a 64 MB shared-memory sub-histogram cannot apply: the cost model
    assert ds.plan_histogram(1 << 27, 1 << 24, 4, 2) == model[(1 << 27, 1 << 24, 4, 2)]
    # regime 0 in an entry: the cost model at that shape
    assert ds.plan_histogram(1 << 27, 1 << 16, 4, 0) == model[(1 << 27, 1 << 16, 4, 0)]
    # too far from every entry (2^12 keys, 2^26 bins): the cost model
    assert ds.plan_histogram(1 << 12, 1 << 26, 4, 2) == model[(1 << 12, 1 << 26, 4, 2)]


def test_forced_fields_bypass_the_table(ds, tmp_path):
    ds.tune_table_load(_write(tmp_path))
    p = ds.plan_histogram(1 << 20, 1 << 8, 4, 2, replicas=2)
    assert p["replicas"] == 2 and p["crn"] == 3  # the cost model with the forced field, not the entry


def test_skew_hint_range(ds):
    with pytest.raises(ds.DialSortError):
        ds.plan_histogram(1 << 20, 1 << 8, 4, 4)


def test_environment_variable_names_the_table(ds, tmp_path):
    path = _write(tmp_path)
    code = "import paper_2605_16667_gb300 as ds; print(ds.tune_table_size())"
    for value, want in ((path, 8), ("", 0)):
        env = dict(os.environ, DIALSORT_TUNE_CACHE=value, PYTHONPATH=ROOT)
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        assert out.returncode == 0, out.stderr
        assert int(out.stdout.split()[-1]) == want


def test_shipped_table_is_well_formed(ds):
    if not os.path.exists(ds.TUNE_TABLE):
        pytest.skip("no measured table shipped")
    n = 0
    with open(ds.TUNE_TABLE) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            lg_n, lg_u, width, skew, regime, crn, rep, threads, per_sm = map(int, line.split())
            assert width in (2, 4) and 0 <= skew <= 3 and regime in (0, 1, 2, 4, 5, 6) and 0 <= crn <= 3
            assert threads in (0, 256, 512, 1024) and per_sm in (0, 1, 2, 4) and rep in (0, 1, 2, 4, 8, 16, 32)
            if width == 2:
                assert lg_u <= 16
            n += 1
    ds.tune_table_load(ds.TUNE_TABLE)
    assert ds.tune_table_size() == n
