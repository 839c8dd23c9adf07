"""The host-core Smoothed Striding yardstick (yardstick/cpu_smoothed.c,
libcpuyard.so), no GPU: the split, the postcondition and the multiset on
sizes that take its serial path (below 2^16 keys) and its OpenMP path, with
one and several threads, pivots at both extremes, and duplicate-heavy keys.
It is timed beside the GPU path by the bench, so it must partition."""
import ctypes
import os

import numpy as np
import pytest

from paper_2004_12532_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2004_12532_gb300", "libcpuyard.so")


@pytest.fixture(scope="module")
def cy():
    from paper_2004_12532_gb300 import build
    try:
        build.build()
    except RuntimeError:
        pass  # the yardstick is optional; the skip below says so
    if not os.path.exists(LIB):
        pytest.skip("libcpuyard.so not built (no OpenMP compiler)")
    L = ctypes.CDLL(LIB)
    L.cy_smoothed_partition_u64.restype = ctypes.c_uint64
    L.cy_smoothed_partition_u64.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                            ctypes.c_int, ctypes.c_uint64]
    return L


@pytest.mark.parametrize("n", [0, 1, 5000, (1 << 16) - 1, (1 << 16) + 3, 1 << 20, 3_000_017])
@pytest.mark.parametrize("threads", [1, 4])
@pytest.mark.parametrize("q", [(1, 100), (1, 2), (99, 100)])
def test_partition(cy, n, threads, q):
    a = inputs.uniform_u64(n, 11 * n + threads)
    pv = inputs.quantile_pivot(*q)
    w = a.copy()
    t = cy.cy_smoothed_partition_u64(w.ctypes.data if n else None, n, pv, threads, 7)
    p = np.uint64(pv)
    assert t == int(np.count_nonzero(a <= p))
    assert np.all(w[:t] <= p) and np.all(w[t:] > p)
    assert np.array_equal(np.sort(w), np.sort(a))


def test_duplicates(cy):
    n = 1 << 20
    a = inputs.uniform_u64(n, 3) % np.uint64(4)
    w = a.copy()
    t = cy.cy_smoothed_partition_u64(w.ctypes.data, n, 1, 4, 1)
    assert t == int(np.count_nonzero(a <= 1))
    assert np.all(w[:t] <= 1) and np.all(w[t:] > 1)
    assert np.array_equal(np.sort(w), np.sort(a))
