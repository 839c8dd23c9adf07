"""Pins of the oracle's Blocked-Prefix-Sum partition (Sec. 3).

Lemma 3.1 (every prefix successor-heavy after preprocessing) by brute force,
the block prefix values against numpy's cumulative sum, and the final
postcondition of the whole low-space partition on both role-swap paths.
"""
import itertools

import numpy as np
import pytest

from paper_2004_12532_gb300 import inputs


def rows(length, alphabet=(1, 2, 3, 4)):
    return [np.array(r, dtype=np.uint64) for r in itertools.product(alphabet, repeat=length)]


@pytest.mark.parametrize("length", range(1, 9))
def test_successor_heavy_bruteforce(orc, length):
    """Lemma 3.1: with successors at least half of A, after the preprocessing
    phase every t-prefix holds at least t/4 successors."""
    for pivot in range(0, 5):
        for r in rows(length):
            if 2 * int((r > pivot).sum()) < length:
                continue
            a = r.copy()
            orc.make_successor_heavy(a, pivot, 0)
            assert np.array_equal(np.sort(a), np.sort(r))
            succ = np.cumsum(a > pivot)
            t = np.arange(1, length + 1)
            assert np.all(4 * succ >= t)


def test_successor_heavy_flipped(orc):
    """Role swap: on the reversed array with dec' = [x > pivot] the same lemma
    holds for the swapped roles."""
    a0 = inputs.uniform_u64(5001, 3)
    p = inputs.quantile_pivot(9, 10)  # predecessors are the majority
    a = a0.copy()
    orc.make_successor_heavy(a, p, 1)
    rev = a[::-1]
    succ_prime = np.cumsum(rev <= np.uint64(p))  # successors of the flipped view
    t = np.arange(1, a.size + 1)
    assert np.all(4 * succ_prime >= t)


@pytest.mark.parametrize("n,B", [(1000, 7), (4096, 64), (5000, 4096), (99, 100)])
def test_block_prefix_cumsum(orc, n, B):
    a = inputs.uniform_u64(n, n)
    p = inputs.quantile_pivot(1, 2)
    v = orc.block_prefix(a, p, B)
    nb = n // B
    assert v.size == nb
    if nb:
        d = (a <= np.uint64(p)).astype(np.int64)
        per_block = [d[i * B:(i + 1) * B].sum() for i in range(nb - 1)]
        per_block.append(d[(nb - 1) * B:].sum())  # last block takes the remainder
        assert np.array_equal(v.astype(np.int64), np.cumsum(per_block))


@pytest.mark.parametrize("length", range(0, 9))
def test_lowspace_bruteforce(orc, length):
    for pivot in range(0, 5):
        for r in rows(length) if length else [np.zeros(0, np.uint64)]:
            for B in (1, 2):
                a = r.copy()
                t = orc.lowspace_partition(a, pivot, B)
                assert t == int((r <= pivot).sum())
                assert np.all(a[:t] <= pivot) and np.all(a[t:] > pivot)
                assert np.array_equal(np.sort(a), np.sort(r))


@pytest.mark.parametrize("q", [(1, 100), (1, 2), (99, 100), (0, 1), (1, 1)])
@pytest.mark.parametrize("B", [4, 64, 4096])
def test_lowspace_random(orc, q, B):
    n = 200003
    a0 = inputs.uniform_u64(n, 77)
    p = inputs.quantile_pivot(*q) if q[0] else 0
    a = a0.copy()
    t = orc.lowspace_partition(a, p, B)
    assert t == int((a0 <= np.uint64(p)).sum())
    assert np.all(a[:t] <= np.uint64(p)) and np.all(a[t:] > np.uint64(p))
    assert np.array_equal(np.sort(a), np.sort(a0))


def test_reorder_after_preprocessing(orc):
    """The three phases called one by one give the partition."""
    n, B = 30000, 16
    a0 = inputs.uniform_u64(n, 5)
    p = inputs.quantile_pivot(2, 5)
    a = a0.copy()
    orc.make_successor_heavy(a, p, 0)
    v = orc.block_prefix(a, p, B)
    orc.reorder(a, p, B, v)
    t = int((a0 <= np.uint64(p)).sum())
    assert np.all(a[:t] <= np.uint64(p)) and np.all(a[t:] > np.uint64(p))
    assert np.array_equal(np.sort(a), np.sort(a0))
