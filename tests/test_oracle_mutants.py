"""The oracle's pins must catch plausible mistakes in the oracle itself.

Each case below plants one mistake (a dropped term, an off-by-one index, a
wrong order, a missing sign flip, ...) in a temporary copy of the oracle's C
source, and runs the pin suite (test_oracle_pins.py) against that copy in a
child process: at least one pin has to fail, by assertion, not by a crash.
A control run on the unmodified copy has to pass, so a failure is the
mistake's doing and not the harness's.  CPU only; nothing here touches the
CUDA path.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

PLACE = ("      uint32_t d = (src[i] >> (8 * pass)) & 255u;\n"
         "      if (is_signed && pass == 3) d = d ^ 0x80u;\n"
         "      dst[cursor[d]] = src[i];")

# name -> (passage the mistake breaks, [(old, new, occurrences to replace: 1 = first only, 0 = all)])
MUTANTS = {
    "histogram adds two per key": ("Eq. (1)", [("H[x] = H[x] + 1;", "H[x] = H[x] + 2;", 1)]),
    "histogram counts x into bin x - 1": ("Eq. (1)", [
        ("H[x] = H[x] + 1;", "H[x ? x - 1 : 0] = H[x ? x - 1 : 0] + 1;", 1)]),
    "histogram drops the last key": ("Eq. (1)", [
        ("for (uint64_t i = 0; i < n; ++i) {\n    uint32_t x = keys[i];",
         "for (uint64_t i = 0; i + 1 < n; ++i) {\n    uint32_t x = keys[i];", 1)]),
    "histogram counts out-of-range keys in the last bin": ("Eq. (1), keys in [0, U)", [
        ("    if (x < U)\n      H[x] = H[x] + 1;",
         "    if (U > 0)\n      H[x < U ? x : U - 1] = H[x < U ? x : U - 1] + 1;", 1)]),
    "projection emits each key one time too few": ("Eq. (2)", [
        ("for (uint64_t j = 0; j < H[k]; ++j) {\n      if (pos < cap) out[pos] = (uint32_t)k;",
         "for (uint64_t j = 1; j < H[k]; ++j) {\n      if (pos < cap) out[pos] = (uint32_t)k;", 1)]),
    "projection walks the bins downward": ("Eq. (2), k ascending", [
        ("  for (uint64_t k = 0; k < U; ++k) {\n    for (uint64_t j = 0; j < H[k]; ++j) {\n"
         "      if (pos < cap) out[pos] = (uint32_t)k;",
         "  for (uint64_t kk = 0; kk < U; ++kk) {\n    uint64_t k = U - 1 - kk;\n"
         "    for (uint64_t j = 0; j < H[k]; ++j) {\n      if (pos < cap) out[pos] = (uint32_t)k;", 1)]),
    "projection emits k + 1": ("Eq. (2)", [("out[pos] = (uint32_t)k;", "out[pos] = (uint32_t)(k + 1);", 1)]),
    "offsets are inclusive sums": ("Eq. (2), the cursor on reaching k", [
        ("    O[k] = cursor;\n    cursor = cursor + H[k];", "    cursor = cursor + H[k];\n    O[k] = cursor;", 1)]),
    "CRN merges distinct keys": ("Eqs. (3)-(4)", [("if (key_in[i] == key_in[i + 1]) {", "if (1) {", 1)]),
    "CRN loses the odd residual": ("Definition \"CRN level transition\"", [
        ("if (i < m) { /* odd residual */", "if (0) { /* odd residual */", 1)]),
    "CRN merge drops the second count": ("Eq. (3)", [
        ("cnt_out[w] = cnt_in[i] + cnt_in[i + 1];", "cnt_out[w] = cnt_in[i];", 1)]),
    "radix takes the most significant digit first": ("Sec. \"Full int32 range\", LSD order", [
        ("(src[i] >> (8 * pass))", "(src[i] >> (8 * (3 - pass)))", 0)]),
    "radix treats int32 as unsigned": ("Sec. \"Full int32 range\", signed keys", [
        ("      if (is_signed && pass == 3) d = d ^ 0x80u;\n", "", 0)]),
    "radix placement is not stable": ("Sec. \"Full int32 range\", stable passes", [
        ("    for (uint64_t i = 0; i < n; ++i) {\n" + PLACE,
         "    for (uint64_t ii = 0; ii < n; ++ii) {\n      uint64_t i = n - 1 - ii;\n" + PLACE, 1)]),
    "range count excludes b": ("Sec. \"Canonical ordered state\", range-count", [
        ("k <= b[i] && k < U", "k < b[i] && k < U", 1)]),
    "presence is true for empty bins": ("Sec. \"Canonical ordered state\", presence", [
        ("H[q[i]] > 0", "H[q[i]] >= 0", 1)]),
    "frequency reads the next bin": ("Sec. \"Canonical ordered state\", frequency", [
        ("freq[i] = q[i] < U ? H[q[i]] : 0;", "freq[i] = q[i] + 1 < U ? H[q[i] + 1] : 0;", 1)]),
    "mapped sort emits indices, not phi_inv": ("Prop. \"General Self-Indexing Principle\"", [
        ("const uint32_t value = phi_inv != 0 ? phi_inv[i] : (uint32_t)i;", "const uint32_t value = (uint32_t)i;", 1)]),
    "accumulate zeroes H first": ("Eq. (1) without the zeroing", [
        ("uint64_t oracle_accumulate_u32(const uint32_t* keys, uint64_t n, uint32_t U, uint32_t* H) {\n",
         "uint64_t oracle_accumulate_u32(const uint32_t* keys, uint64_t n, uint32_t U, uint32_t* H) {\n"
         "  for (uint64_t k = 0; k < U; ++k) H[k] = 0;\n", 1)]),
}


def _mutate(src: str, edits) -> str:
    for old, new, count in edits:
        found = src.count(old)
        assert found >= 1, f"mutation site not found: {old[:60]!r}"
        src = src.replace(old, new) if count == 0 else src.replace(old, new, count)
    return src


def _run_pins(workdir: str, name: str, edits) -> tuple[int, str]:
    """Copy the oracle package into workdir/<name>/oracle with the edits applied, then run the pin suite
    against it in a child process (the copy shadows the real oracle on sys.path)."""
    base = os.path.join(workdir, name.replace(" ", "_").replace(",", ""))
    pkg = os.path.join(base, "oracle")
    os.makedirs(pkg)
    shutil.copy(os.path.join(ORACLE, "__init__.py"), pkg)
    with open(os.path.join(ORACLE, "dialsort_oracle.c")) as f:
        src = f.read()
    with open(os.path.join(pkg, "dialsort_oracle.c"), "w") as f:
        f.write(_mutate(src, edits))
    boot = ("import sys; sys.path[:0] = [sys.argv[1], sys.argv[2]]; import pytest; "
            "sys.exit(pytest.main(['-x', '-q', '-p', 'no:cacheprovider', sys.argv[3]]))")
    r = subprocess.run([sys.executable, "-c", boot, base, ROOT, PINS], capture_output=True, text=True,
                       cwd=base, timeout=600)
    return r.returncode, r.stdout + r.stderr


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc is needed to build the oracle copies")
    work = str(tmp_path_factory.mktemp("oracle_mutants"))
    cases = {"control": []} | {k: v[1] for k, v in MUTANTS.items()}
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        futs = {name: ex.submit(_run_pins, work, name, edits) for name, edits in cases.items()}
        return {name: f.result() for name, f in futs.items()}


def test_control_copy_passes_every_pin(outcomes):
    rc, out = outcomes["control"]
    assert rc == 0, out[-2000:]


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistake_fails_a_pin(outcomes, name):
    rc, out = outcomes[name]
    assert rc != 0, f"the pins did not catch: {name} ({MUTANTS[name][0]})"
    # exit status 1: a pin failed its assertion (a crash, a build or collection error gives another status)
    assert rc == 1 and " failed" in out, out[-2000:]
