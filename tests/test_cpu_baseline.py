"""The benchmark's multi-threaded CPU DialSort (a host throughput line, not the oracle) sorts like the
oracle on every distribution, with keys outside the universe skipped."""
import numpy as np
import pytest

import gen
import oracle

cpu_baseline = pytest.importorskip("cpu_baseline")


@pytest.mark.parametrize("dist", ["uniform", "zipf", "all_equal", "sorted", "runs"])
@pytest.mark.parametrize("threads", [1, 3, 0])
def test_parallel_cpu_dialsort_matches_oracle(dist, threads):
    U = 5000
    keys = gen.keys(300_007, U, dist, stream=830)
    np.testing.assert_array_equal(cpu_baseline.sort(keys, U, threads=threads), oracle.sort(keys, U))


def test_parallel_cpu_dialsort_edges():
    assert cpu_baseline.sort(np.zeros(0, dtype=np.uint32), 10).size == 0
    keys = np.array([3, 12, 0, 3, 9], dtype=np.uint32)  # 12 is outside [0, 10)
    np.testing.assert_array_equal(cpu_baseline.sort(keys, 10, threads=4), [0, 3, 3, 9])
    one = np.full(1000, 7, dtype=np.uint32)
    np.testing.assert_array_equal(cpu_baseline.sort(one, 8, threads=16), one)
