"""Pins for the CPU oracle against what the paper and the mathematics fix.

None of these checks retypes the oracle's own loop: each compares it with a
value the paper prints (tests/golden), brute force over every tiny input, a
library routine (sorted, numpy sort/cumsum/bincount), or an invariant of
Theorem "Correctness of DialSort" / Lemma "CRN additive conservation".
"""
import collections
import itertools
import math

import numpy as np
import pytest

import gen
import oracle
from conftest import load_golden


# ---------------------------------------------------------------- worked examples

def test_fig_viz_worked_example():
    g = load_golden("fig_viz.txt")
    U = g["U"][0]
    H, skipped = oracle.histogram(np.array(g["keys"], dtype=np.uint32), U)
    assert skipped == 0
    assert H.tolist() == g["H"]
    assert oracle.reconstruct(H, U).tolist() == g["out"]
    assert oracle.sort(np.array(g["keys"], dtype=np.uint32), U).tolist() == g["out"]


@pytest.mark.parametrize("name", ["abacus.txt", "physical.txt"])
def test_projection_worked_examples(name):
    g = load_golden(name)
    U = g["U"][0]
    H = np.array(g["H"], dtype=np.uint32)
    out = oracle.reconstruct(H, U)
    assert out.tolist() == g["out"]
    # ingesting the projected output gives the printed state back
    H2, _ = oracle.histogram(out, U)
    assert H2.tolist() == g["H"]


def test_three_arrivals_of_42():
    g = load_golden("crn_three_42.txt")
    k, c = oracle.crn(g["lanes"])
    assert k.tolist() == g["crn_out_keys"] and c.tolist() == g["crn_out_counts"]
    H, _ = oracle.histogram(np.array(g["lanes"], dtype=np.uint32), g["U"][0])
    assert int(H[42]) == g["H42"][0] and int(H.sum()) == 3


# ---------------------------------------------------------------- brute force

@pytest.mark.parametrize("U", [1, 2, 3, 4])
def test_brute_force_all_tiny_inputs(U):
    """Every key sequence of length 0..6 over [0, U): H against list.count, output against sorted()."""
    for n in range(0, 7):
        for seq in itertools.product(range(U), repeat=n):
            keys = np.array(seq, dtype=np.uint32)
            H, skipped = oracle.histogram(keys, U)
            assert skipped == 0
            assert H.tolist() == [list(seq).count(k) for k in range(U)]
            assert oracle.reconstruct(H, U).tolist() == sorted(seq)


def test_brute_force_u16_matches_u32_widened():
    for n in range(0, 6):
        for seq in itertools.product(range(3), repeat=n):
            a = np.array(seq, dtype=np.uint16)
            H16, _ = oracle.histogram(a, 3)
            H32, _ = oracle.histogram(a.astype(np.uint32), 3)
            assert H16.tolist() == H32.tolist()
            assert oracle.reconstruct(H16, 3, width=2).tolist() == sorted(seq)


# ---------------------------------------------------------------- library routines and invariants

DISTS = ["uniform", "zipf", "all_equal", "sorted", "reverse", "runs", "paper_skew", "zipf_perm"]


@pytest.mark.parametrize("dist", DISTS)
@pytest.mark.parametrize("n,U", [(1000, 1), (4099, 7), (1 << 16, 256), (100_003, 1 << 12), (1 << 20, 1 << 16)])
def test_sort_equals_numpy_sort(dist, n, U):
    keys = gen.keys(n, U, dist, param=4096 if dist == "runs" else None, stream=11)
    out = oracle.sort(keys, U)
    assert out.dtype == np.uint32 and out.size == n  # Theorem "Correctness": length n
    np.testing.assert_array_equal(out, np.sort(keys, kind="stable"))


@pytest.mark.parametrize("dist", ["uniform", "zipf", "all_equal", "paper_skew"])
def test_correctness_theorem_invariants(dist):
    n, U = 200_001, 5000
    keys = gen.keys(n, U, dist, stream=12)
    H, _ = oracle.histogram(keys, U)
    assert int(H.astype(np.uint64).sum()) == n  # sum H = n
    np.testing.assert_array_equal(H, np.bincount(keys, minlength=U).astype(np.uint32))
    out = oracle.reconstruct(H, U)
    assert out.size == n
    assert np.all(out[1:] >= out[:-1])  # nondecreasing
    assert collections.Counter(out.tolist()) == collections.Counter(keys.tolist())  # same multiset


def test_u16_equals_u32_on_widened_keys():
    keys16 = gen.keys(300_007, 1 << 16, "zipf", width=2, stream=13)
    H16, _ = oracle.histogram(keys16, 1 << 16)
    H32, _ = oracle.histogram(keys16.astype(np.uint32), 1 << 16)
    np.testing.assert_array_equal(H16, H32)
    out16 = oracle.reconstruct(H16, 1 << 16, width=2)
    assert out16.dtype == np.uint16
    np.testing.assert_array_equal(out16, np.sort(keys16))


# ---------------------------------------------------------------- special cases

def test_all_equal_is_a_fill():
    keys = np.full(12345, 77, dtype=np.uint32)
    H, _ = oracle.histogram(keys, 100)
    assert int(H[77]) == 12345 and int(H.sum()) == 12345
    assert np.all(oracle.reconstruct(H, 100) == 77)


def test_universe_of_one():
    keys = np.zeros(999, dtype=np.uint32)
    H, _ = oracle.histogram(keys, 1)
    assert H.tolist() == [999]
    assert np.all(oracle.reconstruct(H, 1) == 0)


def test_sorted_input_is_a_fixed_point():
    keys = gen.keys(50_000, 1 << 10, "sorted", stream=14)
    assert np.all(keys[1:] >= keys[:-1])
    np.testing.assert_array_equal(oracle.sort(keys, 1 << 10), keys)


def test_empty_input_and_empty_histogram():
    H, skipped = oracle.histogram(np.zeros(0, dtype=np.uint32), 17)
    assert skipped == 0 and H.tolist() == [0] * 17
    assert oracle.reconstruct(H, 17).size == 0


def test_out_of_range_keys_are_skipped():
    keys = np.array([0, 5, 9, 10, 11, 4_000_000_000, 9], dtype=np.uint32)
    H, skipped = oracle.histogram(keys, 10)
    assert skipped == 3
    np.testing.assert_array_equal(H, np.bincount(keys[keys < 10], minlength=10).astype(np.uint32))


def test_reconstruct_cap_truncates_but_reports_total():
    H = np.array([2, 0, 3], dtype=np.uint32)
    out = oracle.reconstruct(H, 3, cap=4)
    assert out.tolist() == [0, 0, 2, 2]


# ---------------------------------------------------------------- offsets

@pytest.mark.parametrize("dist", ["uniform", "zipf", "all_equal"])
def test_offsets_against_cumsum_and_first_occurrence(dist):
    U = 3000
    keys = gen.keys(77_777, U, dist, stream=15)
    H, _ = oracle.histogram(keys, U)
    O = oracle.offsets(H)
    assert O.size == U + 1 and int(O[0]) == 0 and int(O[U]) == keys.size
    np.testing.assert_array_equal(O[1:], np.cumsum(H.astype(np.uint64)))
    out = oracle.reconstruct(H, U)
    present = np.nonzero(H)[0]
    # the run of each present key starts exactly at its offset
    np.testing.assert_array_equal(np.searchsorted(out, present, side="left"), O[present])


# ---------------------------------------------------------------- CRN (Definition "CRN level transition")

def _totals(keys, counts):
    t = collections.Counter()
    for k, c in zip(np.asarray(keys).tolist(), np.asarray(counts).tolist()):
        t[k] += c
    return t


def test_crn_level_pairs_adjacent_items_only():
    k, c = oracle.crn_level([7, 7, 9, 9], [1, 1, 1, 1])
    assert k.tolist() == [7, 9] and c.tolist() == [2, 2]
    k, c = oracle.crn_level([7, 9, 9, 7], [1, 1, 1, 1])  # (7,9) and (9,7): nothing merges
    assert k.tolist() == [7, 9, 9, 7] and c.tolist() == [1, 1, 1, 1]
    k, c = oracle.crn_level([5, 5, 5], [2, 3, 4])  # odd residual forwarded unchanged
    assert k.tolist() == [5, 5] and c.tolist() == [5, 4]
    k, c = oracle.crn_level([], [])
    assert k.size == 0


@pytest.mark.parametrize("m", list(range(1, 33)))
def test_crn_all_equal_lanes_collapse_in_ceil_log2_levels(m):
    k, c = oracle.crn([3] * m)
    assert k.tolist() == [3] and c.tolist() == [m]
    if m > 2:
        # one level fewer than ceil(log2 m) leaves more than one item
        levels = math.ceil(math.log2(m))
        kk, cc = np.array([3] * m, dtype=np.uint32), np.ones(m, dtype=np.uint64)
        for _ in range(levels - 1):
            kk, cc = oracle.crn_level(kk, cc)
        assert kk.size > 1


def test_crn_alternating_keys_never_merge():
    """(a,b,a,b): no adjacent pair is ever equal, so the literal network forwards all four items.

    The definition's closing sentence says every key survives at most once;
    this input shows the pairing rule alone does not give that, so only the
    additive conservation of the lemma is asserted elsewhere.
    """
    k, c = oracle.crn([1, 2, 1, 2])
    assert k.tolist() == [1, 2, 1, 2] and c.tolist() == [1, 1, 1, 1]


@pytest.mark.parametrize("m", [2, 3, 5, 7, 8, 13, 16, 31, 32])
def test_crn_additive_conservation(m):
    rng = np.random.default_rng(1000 + m)
    for trial in range(200):
        keys = rng.integers(0, 1 + trial % 6, size=m).astype(np.uint32)
        counts = rng.integers(1, 5, size=m).astype(np.uint64)
        before = _totals(keys, counts)
        kk, cc = keys, counts
        for _ in range(math.ceil(math.log2(m))):
            kk, cc = oracle.crn_level(kk, cc)
            assert _totals(kk, cc) == before  # invariant at every level
        kf, cf = oracle.crn(keys, counts)
        assert _totals(kf, cf) == before
        # applying the surviving items to H gives the plain histogram of the lanes
        H = np.zeros(8, dtype=np.uint64)
        np.add.at(H, kf.astype(np.int64), cf)
        np.testing.assert_array_equal(H, np.bincount(keys, weights=counts, minlength=8).astype(np.uint64))


# ---- queries on H (Sec. "Canonical ordered state") and accumulating ingestion

def test_queries_on_the_fig_viz_histogram():
    g = load_golden("fig_viz.txt")
    keys = [int(x) for x in g["keys"]]
    U = int(g["U"][0])
    H, _ = oracle.histogram(np.array(keys, dtype=np.uint32), U)
    q = np.arange(U + 2, dtype=np.uint32)  # includes two keys outside the universe
    np.testing.assert_array_equal(oracle.frequency(H, q), [keys.count(k) for k in q])
    np.testing.assert_array_equal(oracle.presence(H, q), [int(k in keys) for k in q])
    a = np.array([1, 0, 3, 4, 2, 5, 6], dtype=np.uint32)
    b = np.array([3, 5, 3, 4, 1, 9, 9], dtype=np.uint32)
    want = [sum(1 for x in keys if lo <= x <= hi) for lo, hi in zip(a, b)]
    np.testing.assert_array_equal(oracle.range_count(H, a, b), want)
    assert want[:3] == [6, 8, 4]  # keys in [1,3]: 1,1,3,3,3,3; all eight; four 3s


@pytest.mark.parametrize("U", [1, 2, 3, 4])
def test_queries_brute_force_tiny(U):
    """Every key sequence of length <= 4 over [0, U), every query key and every (a, b) in [0, U+1]^2,
    counted from the keys themselves."""
    qs = np.arange(U + 2, dtype=np.uint32)
    pairs = np.array([(a, b) for a in range(U + 2) for b in range(U + 2)], dtype=np.uint32)
    for length in range(5):
        for seq in itertools.product(range(U), repeat=length):
            H, _ = oracle.histogram(np.array(seq, dtype=np.uint32), U)
            assert oracle.frequency(H, qs).tolist() == [seq.count(k) for k in qs]
            assert oracle.presence(H, qs).tolist() == [int(k in seq) for k in qs]
            got = oracle.range_count(H, pairs[:, 0], pairs[:, 1]).tolist()
            assert got == [sum(1 for x in seq if a <= x <= b) for a, b in pairs]


@pytest.mark.parametrize("dist", ["uniform", "zipf", "sorted", "all_equal"])
def test_range_count_equals_searchsorted_on_sorted_keys(dist):
    U, n = 100_000, 300_000
    keys = gen.keys(n, U, dist, stream=801)
    H, _ = oracle.histogram(keys, U)
    s = np.sort(keys)
    a = gen.keys(2000, U + 10, "uniform", stream=802)
    b = gen.keys(2000, U + 10, "uniform", stream=803)
    want = np.where(a <= b, np.searchsorted(s, b, side="right") - np.searchsorted(s, a, side="left"), 0)
    np.testing.assert_array_equal(oracle.range_count(H, a, b), want)
    q = gen.keys(5000, U + 10, "uniform", stream=804)
    cnt = np.bincount(keys, minlength=U + 10)
    np.testing.assert_array_equal(oracle.frequency(H, q), cnt[q])
    np.testing.assert_array_equal(oracle.presence(H, q), (cnt[q] > 0).astype(np.uint8))
    full = oracle.range_count(H, np.array([0]), np.array([U - 1]))
    assert int(full[0]) == n  # sum of H = n (Thm. "Correctness")


def test_accumulate_over_batches_equals_one_histogram():
    U = 5000
    keys = gen.keys(200_001, U, "zipf", stream=805)
    H = np.zeros(U, dtype=np.uint32)
    for lo, hi in [(0, 1), (1, 77_777), (77_777, 77_777), (77_777, 200_001)]:
        H, skipped = oracle.accumulate(keys[lo:hi], U, H)
        assert skipped == 0
    np.testing.assert_array_equal(H, np.bincount(keys, minlength=U))
    H2, skipped = oracle.accumulate(np.array([4999, 5000, 0], dtype=np.uint32), U, H)
    assert skipped == 1 and int(H2[4999]) == int(H[4999]) + 1 and int(H2[0]) == int(H[0]) + 1
    Hw, _ = oracle.accumulate(keys.astype(np.uint16), U, np.zeros(U, dtype=np.uint32))
    np.testing.assert_array_equal(Hw, np.bincount(keys, minlength=U))


# ---- DialSort-Radix (Sec. "Full int32 range")

SPECIAL = [-(2 ** 31), -(2 ** 31) + 1, -65536, -257, -256, -255, -1, 0, 1, 255, 256, 257, 65535, 65536,
           2 ** 24, 2 ** 31 - 1]


def test_radix_brute_force_on_special_values():
    """Every sequence of length <= 3 over values at digit and sign boundaries, against sorted()."""
    vals = SPECIAL[::2] + [7]
    for length in range(4):
        for seq in itertools.product(vals, repeat=length):
            got = oracle.radix_sort(np.array(seq, dtype=np.int32))
            assert got.tolist() == sorted(seq)
    u = [0, 1, 255, 256, 2 ** 31 - 1, 2 ** 31, 2 ** 32 - 1]
    for seq in itertools.product(u, repeat=3):
        assert oracle.radix_sort(np.array(seq, dtype=np.uint32)).tolist() == sorted(seq)


@pytest.mark.parametrize("n", [0, 1, 5, 1000, 100_003])
def test_radix_equals_numpy_sort_full_int32_range(n):
    w = gen.words(n, stream=806)
    signed = w.astype(np.uint32).view(np.int32)
    np.testing.assert_array_equal(oracle.radix_sort(signed), np.sort(signed))
    np.testing.assert_array_equal(oracle.radix_sort(w.astype(np.uint32)), np.sort(w.astype(np.uint32)))


def test_radix_special_cases():
    vals = np.array(SPECIAL * 50, dtype=np.int32)
    np.testing.assert_array_equal(oracle.radix_sort(vals), np.sort(vals))
    same = np.full(1000, -7, dtype=np.int32)
    np.testing.assert_array_equal(oracle.radix_sort(same), same)  # all equal: a fixed point
    asc = np.sort(gen.words(5000, stream=807).astype(np.uint32).view(np.int32))
    np.testing.assert_array_equal(oracle.radix_sort(asc), asc)  # sorted input: a fixed point
    np.testing.assert_array_equal(oracle.radix_sort(asc[::-1].copy()), asc)  # reversed
    small = gen.keys(20_000, 1 << 20, "zipf", stream=808).view(np.int32)  # top digits all zero
    np.testing.assert_array_equal(oracle.radix_sort(small), np.sort(small))


# ---- mapped domains (Prop. "General Self-Indexing Principle")

def test_mapped_identity_examples_of_the_proposition():
    """The proposition's own domains with phi = identity: characters (code points), grayscale
    pixels (U = 256), MIDI notes (U = 128), calendar days (U = 366)."""
    text = b"DIALSORT SORTS WITHOUT COMPARISONS"
    out, H, skipped = oracle.sort_mapped(np.frombuffer(text, dtype=np.uint8), 128)
    assert skipped == 0 and bytes(out) == bytes(sorted(text))
    pixels = gen.keys(50_000, 256, "zipf", stream=809).astype(np.uint8)
    out, H, _ = oracle.sort_mapped(pixels, 256)
    np.testing.assert_array_equal(out, np.sort(pixels))
    np.testing.assert_array_equal(H, np.bincount(pixels, minlength=256))
    notes = gen.keys(3000, 128, "uniform", stream=810).astype(np.uint8)
    np.testing.assert_array_equal(oracle.sort_mapped(notes, 128)[0], np.sort(notes))
    days = gen.keys(4000, 366, "uniform", stream=811).astype(np.uint16)
    np.testing.assert_array_equal(oracle.sort_mapped(days, 366)[0], np.sort(days))


def test_mapped_sparse_domain_through_rank_maps():
    """S = 500 distinct 32-bit values; phi = rank in S, phi_inv = S in order: sorting through the
    index space gives the library sort of the keys."""
    S = np.unique(gen.keys(600, 1 << 24, "uniform", stream=812))[:500]
    M = int(S.max()) + 1
    phi = np.full(M, 0xFFFFFFFF, dtype=np.uint32)
    phi[S] = np.arange(S.size, dtype=np.uint32)
    keys = S[gen.keys(20_000, S.size, "zipf", stream=813)]
    out, H, skipped = oracle.sort_mapped(keys, S.size, phi, S)
    assert skipped == 0
    np.testing.assert_array_equal(out, np.sort(keys))
    bad = keys.copy()
    gap = int(np.setdiff1d(np.arange(M, dtype=np.uint32), S)[0])  # a raw value below M outside S
    bad[:3] = [M + 5, gap, M + 7]
    out2, _, skipped2 = oracle.sort_mapped(bad, S.size, phi, S)
    assert skipped2 == 3 and out2.size == keys.size - 3


def test_mapped_follows_phi_order_not_key_order():
    """A phi that reverses the domain emits the keys in descending raw order."""
    U = 1000
    phi = (U - 1 - np.arange(U)).astype(np.uint32)
    keys = gen.keys(5000, U, "uniform", stream=814)
    out, _, _ = oracle.sort_mapped(keys, U, phi, phi)  # phi is its own inverse
    np.testing.assert_array_equal(out, np.sort(keys)[::-1])
    tiny = [3, 1, 2, 1]
    got = oracle.sort_mapped(np.array(tiny, dtype=np.uint32), 4, np.array([3, 2, 1, 0], dtype=np.uint32),
                             np.array([3, 2, 1, 0], dtype=np.uint32))[0].tolist()
    assert got == sorted(tiny, key=lambda x: 3 - x)
