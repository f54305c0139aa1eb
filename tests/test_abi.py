"""The C ABI library loads and exports every symbol include/*.h declares (no GPU needed)."""
import glob
import os
import re

import pytest

from conftest import ROOT


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        names |= set(re.findall(r"\b(dialsort_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g

    g.build()
    from paper_2605_16667_gb300 import native

    return native.load()


def test_header_declares_entry_points():
    names = _declared()
    for must in ("dialsort_histogram", "dialsort_reconstruct", "dialsort_sort", "dialsort_stream_status"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported by libdialsort.so"


def test_binding_covers_every_declared_symbol():
    from paper_2605_16667_gb300 import native

    missing = [n for n in _declared() if n not in native.SIGNATURES]
    assert not missing, f"binding lacks signatures for {missing}"


def test_host_side_queries_without_gpu(lib):
    assert lib.dialsort_version().startswith(b"dialsort-gb300")
    assert lib.dialsort_status_string(2) == b"a key was outside [0, U) and was not counted"
    assert lib.dialsort_sort_workspace_size(1 << 20, 1 << 16) >= 4 * (1 << 16)
    assert lib.dialsort_reconstruct_workspace_size(1 << 20, 1 << 28) > 0


def test_host_validation_rejects_bad_arguments_before_launch(lib):
    # every one of these is refused on the host, so no device is touched
    assert lib.dialsort_histogram(None, 10, 16, 4096, None) == 1  # null keys with n > 0
    assert lib.dialsort_histogram(4096, 10, 0, 4096, None) == 1  # U = 0
    assert lib.dialsort_histogram(4096, 1 << 32, 16, 4096, None) == 1  # n >= 2^32
    assert lib.dialsort_histogram(4097, 10, 16, 4096, None) == 1  # keys not 4-byte aligned
    assert lib.dialsort_histogram(4096, 10, 16, 4100, None) == 1  # H not 16-byte aligned
    assert lib.dialsort_histogram_u16(4096, 10, 65537, 4096, None) == 1  # u16 keys need U <= 65536
    assert lib.dialsort_sort(4096, 10, 16, 8192, None, 0, None) == 8  # no workspace
    assert lib.dialsort_reconstruct(4096, 16, 8192, 10, 4096, 1, None) == 8  # workspace too small


@pytest.fixture
def cost_model():
    """The planner without a measured table (the cost model alone); the default table afterwards."""
    import paper_2605_16667_gb300 as ds

    ds.tune_table_load(None)
    yield ds
    ds.tune_table_load(ds.TUNE_TABLE if os.path.exists(ds.TUNE_TABLE) else None)


def test_autotuner_plans_without_gpu(cost_model):
    ds = cost_model

    p = ds.plan_histogram(1 << 28, 1 << 8)
    assert p["regime_name"] == "smem32" and p["blocks"] >= 1
    p = ds.plan_histogram(1 << 27, 1 << 16)
    assert p["regime_name"] in ("smem16", "smem32")
    p = ds.plan_histogram(1 << 28, 1 << 20, skew_hint=1)
    assert p["regime_name"] == "two_level"  # what dialsort_sort runs on aligned keys
    p = ds.plan_histogram(1 << 28, 1 << 20, skew_hint=1, regime="global")
    assert p["regime_name"] == "global"
    p = ds.plan_histogram(1 << 20, 1 << 16)
    assert p["regime_name"] == "two_level"  # merging 152 x 2^16-bin sub-histograms would dominate n = 2^20
    p = ds.plan_histogram(1 << 20, 1 << 16, regime="auto", width=2)
    assert p["regime_name"] in ("global", "global_crn")  # 16-bit keys: single-pass L2 regime
    with pytest.raises(ds.DialSortError):
        ds.plan_histogram(1 << 20, 1 << 20, regime="smem32")  # 4 MiB sub-histogram does not fit
