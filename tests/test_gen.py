"""The seeded input generators: ranges, determinism and distribution shapes."""
import numpy as np
import pytest

import gen


@pytest.mark.parametrize("dist", sorted(gen.DISTS))
@pytest.mark.parametrize("width,U", [(4, 1), (4, 1000), (4, 1 << 20), (2, 1 << 16), (2, 300)])
def test_range_and_determinism(dist, width, U):
    a = gen.keys(20_001, U, dist, width=width, stream=3)
    b = gen.keys(20_001, U, dist, width=width, stream=3)
    c = gen.keys(20_001, U, dist, width=width, stream=4)
    assert a.dtype == (np.uint32 if width == 4 else np.uint16)
    assert int(a.max()) < U
    np.testing.assert_array_equal(a, b)
    if U > 1000 and dist != "all_equal":
        assert not np.array_equal(a, c)


def test_shapes():
    U = 1 << 16
    s = gen.keys(100_000, U, "sorted", stream=5)
    assert np.all(np.diff(s.astype(np.int64)) >= 0) and s[-1] > U * 0.9 and s[0] < U * 0.1
    r = gen.keys(100_000, U, "reverse", stream=5)
    np.testing.assert_array_equal(r, s[::-1])
    runs = gen.keys(10_000, U, "runs", param=1000, stream=5)
    for b in range(10):
        blk = runs[b * 1000:(b + 1) * 1000].astype(np.int64)
        assert np.all(np.diff(blk) >= 0) if b % 2 == 0 else np.all(np.diff(blk) <= 0)
    z = gen.keys(1 << 20, 1 << 20, "zipf", param=1.2, stream=5)
    # P(0) = 1 / zeta_U(1.2); zeta(1.2) ~ 5.59 (truncated at 2^20 ~ 5.0) -> about 20 % of keys are 0
    frac0 = float(np.mean(z == 0))
    assert 0.17 < frac0 < 0.23
    zp = gen.keys(1 << 20, 1 << 20, "zipf_perm", param=1.2, stream=5)
    vals, cnt = np.unique(zp, return_counts=True)
    assert 0.17 < cnt.max() / zp.size < 0.23
    ps = gen.keys(1 << 20, 10_000, "paper_skew", stream=5)
    hot = float(np.mean(ps <= 500))  # [0, floor(0.05 U)] inclusive
    assert 0.80 < hot < 0.83  # 0.8 + 0.2 * 501/10000
    eq = gen.keys(1000, 1 << 20, "all_equal", stream=5)
    assert np.all(eq == (0x5A5A5 % (1 << 20)))


def test_loguniform_bounds():
    v = gen.loguniform(100_000, 10, 22, stream=7)
    assert v.min() >= 1 << 10 and v.max() <= 1 << 22
    lg = np.log2(v.astype(np.float64))
    assert abs(lg.mean() - 16.0) < 0.05  # log-uniform: mean exponent (10 + 22) / 2
