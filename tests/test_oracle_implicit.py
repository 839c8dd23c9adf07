"""Pins of the oracle's fully in-place Blocked-Prefix-Sum partition (Sec. 3:
values kept in the order of each block's keys, Lemma bitstore2), against
facts that do not come from the oracle itself:

- the encoding round trip: any value in [0, 2^L) written into 4L + 2 keys
  reads back, after any number of later writes, and the keys it overwrote
  come back on restore (the lemma's two properties);
- the choice of encoding: at least L + 1 unequal pairs give the order
  encoding, otherwise the overwrite encoding, and the wanted pairs keep their
  relative order;
- the prefix phase: after it, block i reads back the number of predecessors
  before it, counted by brute force on the restored array; each block holds
  the same multiset as that block of the explicit MakeSuccessorHeavy result;
- the whole partition: the postcondition, the count, and the multiset.
"""
import numpy as np
import pytest

import oracle
from paper_2004_12532_gb300 import inputs


def _rng(seed):
    return np.random.default_rng(seed)


@pytest.mark.parametrize("L", [1, 2, 5, 17, 31, 40])
def test_bitstore_round_trip_distinct(L):
    r = _rng(L)
    for trial in range(30):
        x = np.unique(r.integers(0, 2**62, size=8 * L + 8, dtype=np.uint64))
        x = r.permutation(x)[:4 * L + 2].copy()
        assert x.size == 4 * L + 2
        orig = x.copy()
        v = int(r.integers(0, 2**L))
        oracle.bitstore_encode(x, L, v, True)
        assert x[0] != x[1]  # distinct keys: the order encoding
        assert np.array_equal(np.sort(x), np.sort(orig))  # only reordered
        assert oracle.bitstore_decode(x, L, restore=False) == v
        for _ in range(3):  # later writes
            v = int(r.integers(0, 2**L))
            oracle.bitstore_encode(x, L, v, False)
            assert oracle.bitstore_decode(x, L, restore=False) == v
        assert oracle.bitstore_decode(x, L, restore=True) == v
        assert np.array_equal(np.sort(x), np.sort(orig))


@pytest.mark.parametrize("L", [1, 3, 31])
def test_bitstore_round_trip_all_equal(L):
    for v in [0, 1, 2**L - 1, (2**L - 1) // 3]:
        x = np.full(4 * L + 2, 12345, dtype=np.uint64)
        oracle.bitstore_encode(x, L, v, True)
        assert x[0] == x[1]  # no unequal pair: the overwrite encoding
        assert oracle.bitstore_decode(x, L, restore=False) == v
        oracle.bitstore_encode(x, L, v ^ 1, False)
        assert oracle.bitstore_decode(x, L, restore=True) == v ^ 1
        assert np.all(x == 12345)  # the overwritten keys are back


@pytest.mark.parametrize("L", [2, 6, 20])
@pytest.mark.parametrize("unequal_extra", [0, 1])
def test_bitstore_choice_boundary(L, unequal_extra):
    """Of 2L + 1 pairs, L + unequal_extra are unequal: L + 1 unequal pairs
    select the order encoding, L select the overwrite encoding."""
    r = _rng(100 + L)
    P = 2 * L + 1
    n_uneq = L + unequal_extra
    which = np.zeros(P, bool)
    which[r.choice(P, n_uneq, replace=False)] = True
    pairs = []
    for k in range(P):
        a = int(r.integers(10, 2**40))
        pairs.append((a, a + 1 + int(r.integers(0, 5))) if which[k] else (a, a))
    x = np.array([y for p in pairs for y in p], dtype=np.uint64)
    orig = x.copy()
    v = int(r.integers(0, 2**L))
    oracle.bitstore_encode(x, L, v, True)
    got = [(int(x[2 * k]), int(x[2 * k + 1])) for k in range(P)]
    order_kind = n_uneq >= L + 1
    assert (got[0][0] != got[0][1]) == order_kind
    # the wanted pairs first, in their original relative order (as sets)
    wanted = [tuple(sorted(p)) for p, w in zip(pairs, which) if w == order_kind]
    if order_kind:
        assert [tuple(sorted(p)) for p in got[:len(wanted)]] == wanted
    else:
        assert [p[0] for p in got[:len(wanted)]] == [p[0] for p in wanted]
    assert oracle.bitstore_decode(x, L, restore=True) == v
    assert np.array_equal(np.sort(x), np.sort(orig))


def _logical(a, flip):
    return a[::-1].copy() if flip else a.copy()


@pytest.mark.parametrize("n", [5000, 20011, 131072 + 77])
@pytest.mark.parametrize("q", [(1, 3), (1, 2), (4, 5)])
@pytest.mark.parametrize("dups", [False, True])
def test_implicit_prefix_values(n, q, dups):
    L = oracle.bits_for(n)
    B = 4 * L + 2 + 7
    a = inputs.uniform_u64(n, n + q[0])
    if dups:
        a = a % np.uint64(5)  # mostly equal pairs: the overwrite encoding
        pv = 1
    else:
        pv = inputs.quantile_pivot(*q)
    work = a.copy()
    t, flip = oracle.implicit_prefix(work, pv, B)
    assert t == int(np.count_nonzero(a <= np.uint64(pv)))
    assert flip == (1 if 2 * (n - t) < n else 0)
    view = _logical(work, flip)
    nb = n // B
    vals = [oracle.bitstore_decode(view[i * B:i * B + 4 * L + 2], L, restore=True)
            for i in range(nb)]
    # view is now restored: brute-force predecessor counts per block
    isp = (view > np.uint64(pv)) if flip else (view <= np.uint64(pv))
    ends = [(i + 1) * B if i + 1 < nb else n for i in range(nb)]
    before = 0
    for i in range(nb):
        assert vals[i] == before, (i, vals[i], before)
        before += int(np.count_nonzero(isp[i * B:ends[i]]))
    # the blocks hold the explicit MakeSuccessorHeavy arrangement's multisets
    ref = a.copy()
    oracle.make_successor_heavy(ref, pv, flip)
    rview = _logical(ref, flip)
    for i in range(nb):
        s, e = i * B, ends[i]
        assert np.array_equal(np.sort(view[s:e]), np.sort(rview[s:e]))


@pytest.mark.parametrize("n", [1, 2, 3, 200, 5000, 65536 + 3, 300007])
@pytest.mark.parametrize("kind", ["uniform", "dup4", "sorted"])
@pytest.mark.parametrize("q", [(1, 100), (1, 2), (99, 100)])
def test_implicit_partition(n, kind, q):
    L = oracle.bits_for(n)
    B = max(4 * L + 2, 64)
    a = inputs.uniform_u64(n, 3 * n + q[0])
    pv = inputs.quantile_pivot(*q)
    if kind == "dup4":
        a = a % np.uint64(4)
        pv = 1
    elif kind == "sorted":
        a = np.sort(a)
    work = a.copy()
    t = oracle.implicit_partition(work, pv, B)
    p = np.uint64(pv)
    assert t == int(np.count_nonzero(a <= p))
    assert np.all(work[:t] <= p) and np.all(work[t:] > p)
    assert np.array_equal(np.sort(work), np.sort(a))


def test_bits_for_is_the_bit_length():
    """L = ceil(log2(n + 1)), the bits of a value in [0, n]: the bit length of
    n (Python's int.bit_length, an independent definition), at the powers of
    two and their neighbours and at random sizes."""
    r = _rng(5)
    cases = [0, 1, 2, 3, 4, 5, 7, 8, 9] + [(1 << k) + d for k in range(1, 63) for d in (-1, 0, 1)]
    cases += [int(x) for x in r.integers(0, 2**62, size=200)]
    for n in cases:
        assert oracle.bits_for(n) == n.bit_length(), n
        # the smallest L with n < 2^L, i.e. ceil(log2(n + 1))
        assert n < (1 << oracle.bits_for(n)) and (n == 0 or n >= (1 << (oracle.bits_for(n) - 1)))
