"""Pins of the CPU oracle against facts the paper and mathematics fix.

Nothing here compares the oracle with itself: each check is a closed form,
an invariant stated by the paper, a brute-force enumeration, a golden vector
or a library routine (numpy sort / cumsum / bincount) on a special case.
"""
import itertools
import os

import numpy as np
import pytest

from paper_2004_12532_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def all_arrays(length, alphabet=(1, 2, 3, 4)):
    if length == 0:
        return np.zeros((1, 0), dtype=np.uint64)
    rows = np.array(list(itertools.product(alphabet, repeat=length)), dtype=np.uint64)
    return np.ascontiguousarray(rows)


# ---------------------------------------------------------------- generator
def test_splitmix64_golden(orc):
    vals = [int(x) for x in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if x.strip() and not x.startswith("#")]
    seed, expect = vals[0], vals[1:]
    got = [orc.stream(seed, k) for k in range(len(expect))]
    assert got == expect
    # the numpy input generator implements the same published definition
    assert [int(x) for x in inputs.splitmix_outputs(seed, 0, len(expect))] == expect


def test_range_closed_form(orc):
    rs = [0, 1, 2**63, 2**64 - 1, 0x123456789ABCDEF0, 0xFEDCBA9876543210]
    for r in rs:
        for g in [1, 2, 3, 7, 152, 1000003, 2**32 + 5]:
            assert orc.rng_range(r, g) == (r * g) >> 64  # exact big-int form
            assert 0 <= orc.rng_range(r, g) < g


def test_quantile_pivots():
    assert inputs.quantile_pivot(1, 2) == 2**63 - 1  # "key < 2^63"
    assert inputs.quantile_pivot(1, 100) == -(-(2**64) // 100) - 1
    assert inputs.quantile_pivot(99, 100, 32) == -(-(99 * 2**32) // 100) - 1


# ---------------------------------------------------------------- partition
@pytest.mark.parametrize("length", range(0, 9))
def test_partition_bruteforce(orc, length):
    """Every array of length <= 8 over {1,2,3,4}, every pivot 0..4: the
    postcondition of the problem (Sec. 2), permutation, and t = count."""
    base = all_arrays(length)
    for pivot in range(0, 5):
        a = base.copy()
        t = orc.partition_rows(a, pivot).astype(np.int64)
        cnt = (base <= pivot).sum(axis=1)
        assert np.array_equal(t, cnt)
        idx = np.arange(length)[None, :]
        left = idx < t[:, None]
        assert np.all((a <= pivot) == left)
        assert np.array_equal(np.sort(a, axis=1), np.sort(base, axis=1))


def test_partition_random_sizes(orc):
    for n, seed in [(1, 1), (2, 2), (1000, 3), (100003, 4)]:
        a = inputs.uniform_u64(n, seed)
        ref = a.copy()
        p = inputs.quantile_pivot(1, 2)
        t = orc.partition(a, p)
        assert t == int((ref <= np.uint64(p)).sum())
        assert np.all(a[:t] <= np.uint64(p)) and np.all(a[t:] > np.uint64(p))
        assert np.array_equal(np.sort(a), np.sort(ref))


def test_partition_u32(orc):
    a = inputs.uniform_u32(50001, 9)
    ref = a.copy()
    p = inputs.quantile_pivot(1, 4, 32)
    t = orc.partition(a, p)
    assert t == int((ref <= p).sum())
    assert np.all(a[:t] <= p) and np.all(a[t:] > p)
    assert np.array_equal(np.sort(a), np.sort(ref))


def test_partition_kv_moves_payload(orc):
    k = inputs.uniform_u64(20000, 11)
    v = np.arange(k.size, dtype=np.uint64)
    k0 = k.copy()
    p = inputs.quantile_pivot(3, 10)
    t = orc.partition_kv(k, v, p)
    assert t == int((k0 <= np.uint64(p)).sum())
    assert np.array_equal(k0[v.astype(np.int64)], k)  # payload i still names key i
    assert np.all(k[:t] <= np.uint64(p)) and np.all(k[t:] > np.uint64(p))


def test_partition_extreme_pivots(orc):
    a = inputs.uniform_u64(1000, 5)
    assert orc.partition(a.copy(), 2**64 - 1) == 1000
    b = a.copy()
    assert orc.partition(b, 0) == int((a == 0).sum())


# ---------------------------------------------------------------- quicksort
@pytest.mark.parametrize("length", range(0, 9))
def test_quicksort_bruteforce_vs_counting_sort(orc, length):
    base = all_arrays(length)
    for r in range(base.shape[0]):
        a = base[r].copy()
        orc.quicksort(a, seed=r)
        counts = np.bincount(base[r].astype(np.int64), minlength=5)
        expect = np.repeat(np.arange(5, dtype=np.uint64), counts)
        assert np.array_equal(a, expect)


@pytest.mark.parametrize("kind", ["uniform", "sorted", "reverse", "dup16", "zeros"])
def test_quicksort_vs_numpy(orc, kind):
    n = 200003
    if kind == "uniform":
        a = inputs.uniform_u64(n, 21)
    elif kind == "sorted":
        a = inputs.sorted_u64(n, 22)
    elif kind == "reverse":
        a = inputs.reverse_sorted_u64(n, 23)
    elif kind == "dup16":
        a = inputs.heavy_duplicates_u64(n, 24)
    else:
        a = np.zeros(n, dtype=np.uint64)
    expect = np.sort(a)
    orc.quicksort(a, seed=7)
    assert np.array_equal(a, expect)


def test_quicksort_u32(orc):
    a = inputs.uniform_u32(100001, 31)
    expect = np.sort(a)
    orc.quicksort(a, seed=3)
    assert np.array_equal(a, expect)


# ---------------------------------------------------------------- count
def test_count_is_the_predicate_count(orc):
    """t = #{x <= pivot} (Sec. 2's decider), against numpy's count on random
    keys of both widths, at pivots that hit a key, miss every key, and sit at
    the extremes."""
    r = np.random.default_rng(9)
    for n in [0, 1, 2, 17, 1000, 65537]:
        a64 = r.integers(0, 2**64, size=n, dtype=np.uint64)
        a32 = r.integers(0, 2**32, size=n, dtype=np.uint32)
        piv64 = [0, 2**64 - 1, 2**63] + ([int(a64[n // 2])] if n else [])
        piv32 = [0, 2**32 - 1, 2**31] + ([int(a32[n // 2])] if n else [])
        for p in piv64:
            assert orc.count(a64, p) == int(np.count_nonzero(a64 <= np.uint64(p)))
        for p in piv32:
            assert orc.count(a32, p) == int(np.count_nonzero(a32 <= np.uint32(p)))
