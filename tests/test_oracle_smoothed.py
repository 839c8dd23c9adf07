"""Pins of the oracle's Smoothed Striding and Strided routines (Sec. 4).

Checks are facts the paper states or derives: the partially-partitioned
invariant after the Partial Partition Step, the location of each v_i, the
special cases g = 1 and sorted input, the concentration bound of
Proposition 4.2 (via the Hoeffding step of its proof), and the paper's remark
that the Strided Algorithm makes no progress on inputs aligned to its stride
while the random offsets X do.
"""
import math

import numpy as np
import pytest

from paper_2004_12532_gb300 import inputs

P50 = inputs.quantile_pivot(1, 2)


def line_groups(n, b, g, X):
    """Group index of every line, by inverting 'line j*g + (X[j]+i) mod g of
    chunk j belongs to U_i': i = (line mod g - X[j]) mod g."""
    L = -(-n // b)
    lines = np.arange(L, dtype=np.int64)
    j = lines // g
    return (lines % g - X[j].astype(np.int64)) % g


def check_step(orc, a0, pivot, b, g, X):
    a = a0.copy()
    k, v, vmin, vmax = orc.smoothed_step(a, pivot, b, g, X)
    n = a.size
    pred0 = a0 <= pivot
    pred = a <= pivot
    # permutation of the array
    assert np.array_equal(np.sort(a), np.sort(a0))
    # partially partitioned: A[p] predecessor for p < vmin, successor p >= vmax
    assert np.all(pred[:vmin]) and not np.any(pred[vmax:])
    assert 0 <= vmin <= vmax <= n
    # every group keeps its own multiset and ends predecessors-first
    grp_of_line = line_groups(n, b, g, X)
    grp = np.repeat(grp_of_line, b)[:n]
    for i in range(g):
        sel = np.nonzero(grp == i)[0]  # slots of U_i in increasing position
        if sel.size == 0:
            continue
        assert np.array_equal(np.sort(a[sel]), np.sort(a0[sel]))
        ki = int(pred0[sel].sum())
        assert int(k[i]) == ki
        assert np.all(pred[sel[:ki]]) and not np.any(pred[sel[ki:]])
        expect_v = sel[ki] if ki < sel.size else sel[-1] + 1
        assert int(v[i]) == expect_v
    return a, k, v, vmin, vmax


@pytest.mark.parametrize("n,b,g", [(4096, 8, 16), (5000, 8, 16), (777, 5, 7),
                                   (1 << 14, 64, 32), (100, 128, 4), (0, 4, 3),
                                   (3, 4, 5)])
def test_step_invariants(orc, n, b, g):
    a0 = inputs.uniform_u64(n, 100 + n)
    s = orc.num_chunks(n, b, g)
    X = orc.draw_X(7, 0, s, g)
    check_step(orc, a0, P50, b, g, X)


@pytest.mark.parametrize("n,b,g,q", [(10000, 16, 24, (1, 3)), (4099, 8, 7, (1, 2)),
                                     (1 << 13, 32, 16, (99, 100)), (777, 5, 9, (1, 100))])
def test_step_u32(orc, n, b, g, q):
    """The 4-byte step against the same per-group facts as the 8-byte one:
    each U_i keeps its multiset, ends predecessors-first, and reports its own
    k_i and v_i.  Keys span the whole 32-bit range (half of them have the top
    bit set), so a signed or narrowed compare would miscount some group."""
    a0 = inputs.uniform_u32(n, 3 + n)
    assert np.any(a0 >= np.uint32(1 << 31))
    X = orc.draw_X(5, 2, orc.num_chunks(n, b, g), g)
    check_step(orc, a0, inputs.quantile_pivot(q[0], q[1], 32), b, g, X)


def test_v_locality(orc):
    """Sec. 4 proof of Prop. 4.2: slot k_i of U_i lies in U_i's
    ceil(s*mu_i)-th line, so v_i lies in chunk floor(k_i/b), and
    |v_i - n*mu_i| <= g*b with mu_i = k_i/|U_i| (all lines real)."""
    b, g, s = 16, 32, 64
    n = b * g * s
    for seed in range(5):
        a0 = inputs.uniform_u64(n, 40 + seed)
        X = orc.draw_X(seed, 0, s, g)
        a = a0.copy()
        k, v, vmin, vmax = orc.smoothed_step(a, P50, b, g, X)
        for i in range(g):
            ki = int(k[i])
            if ki < s * b:
                assert int(v[i]) // (g * b) == ki // b
            mu = ki / (s * b)
            assert abs(int(v[i]) - n * mu) <= g * b


def test_g1_is_serial_partition(orc):
    """g = 1: one group holding every line in order, i.e. a plain partition
    (the paper's base case); vmin = vmax = t."""
    a0 = inputs.uniform_u64(3001, 8)
    a = a0.copy()
    k, v, vmin, vmax = orc.smoothed_step(a, P50, 10, 1, np.zeros(301, np.uint64))
    t = int((a0 <= np.uint64(P50)).sum())
    assert vmin == vmax == t == int(k[0])
    assert np.all(a[:t] <= np.uint64(P50)) and np.all(a[t:] > np.uint64(P50))


def test_sorted_input_marker(orc):
    """a[p] = p: each U_i visits positions in increasing order, so every group
    is already partitioned and the step moves nothing; v_i is U_i's first
    position above the pivot.  The expected vmin/vmax follow from the chunk
    geometry alone: the chunk holding the pivot position decides."""
    b, g, s = 4, 8, 16
    n = b * g * s
    a0 = np.arange(n, dtype=np.uint64)
    X = orc.draw_X(3, 0, s, g)
    for P in [0, 5, 31, 32, 200, n - 2]:
        a = a0.copy()
        k, v, vmin, vmax = orc.smoothed_step(a, P, b, g, X)
        assert np.array_equal(a, a0)
        jstar = P // (g * b)                     # chunk containing position P
        chunk0 = jstar * g * b
        firsts = []
        for i in range(g):
            line_in = (int(X[jstar]) + i) % g    # U_i's line inside that chunk
            start = chunk0 + line_in * b
            if start > P:
                firsts.append(start)
            elif start + b - 1 > P:
                firsts.append(P + 1)
            elif jstar + 1 < s:                  # next chunk's line of U_i
                firsts.append((jstar + 1) * g * b + ((int(X[jstar + 1]) + i) % g) * b)
            else:                                # U_i has no successor
                firsts.append(start + b)
        assert vmin == min(firsts)
        if P + 1 < (s - 1) * g * b:
            assert vmin == P + 1
        assert vmax == max(firsts)


def hoeffding_delta(n, b, s, eps):
    # Prop. 4.2's proof: Pr[|mu_i - mu| >= delta] < 2 exp(-2 s delta^2), then a
    # union bound over the groups gives failure probability <= eps.
    return math.sqrt(math.log(2 * n / (b * eps)) / (2 * s))


def test_prop42_concentration(orc):
    """Prop. 4.2: with all |mu_i - mu| < delta, vmax - vmin <= 2n(delta + 1/s).
    Adversarial input: whole lines are predecessors or successors, arranged
    with period g so the Strided Algorithm is at its worst."""
    b, g, s = 8, 64, 512
    n = b * g * s
    eps = 1e-3
    delta = hoeffding_delta(n, b, s, eps)
    bound = 2 * n * (delta + 1.0 / s)
    line = np.arange(n // b)
    pattern = np.where((line % g) < g // 2, np.uint64(0), np.uint64(2**64 - 1))
    a0 = np.repeat(pattern, b)
    worst = 0
    for seed in range(12):
        X = orc.draw_X(1000 + seed, 0, s, g)
        a = a0.copy()
        _, _, vmin, vmax = orc.smoothed_step(a, P50, b, g, X)
        worst = max(worst, vmax - vmin)
        assert vmax - vmin <= bound
    # the Strided Algorithm (X == 0) makes almost no progress on this input
    a = a0.copy()
    _, _, vmin, vmax = orc.smoothed_step(a, P50, b, g, np.zeros(s, np.uint64))
    assert vmax - vmin >= n // 2 - g * b
    assert worst < (vmax - vmin) / 4


def test_X_uniform(orc):
    """X[j] uniform over {0..g-1}: chi-square over many draws."""
    g, s = 10, 20000
    X = orc.draw_X(99, 4, s, g)
    assert X.max() < g
    cnt = np.bincount(X.astype(np.int64), minlength=g)
    chi2 = float(((cnt - s / g) ** 2 / (s / g)).sum())
    assert chi2 < 40.0  # 9 dof; p ~ 1e-5


@pytest.mark.parametrize("kind", ["uniform", "sorted", "period", "dup"])
def test_recursive_smoothed_partition(orc, kind):
    n = 300007
    if kind == "uniform":
        a0 = inputs.uniform_u64(n, 17)
    elif kind == "sorted":
        a0 = inputs.sorted_u64(n, 18)
    elif kind == "period":
        a0 = np.where((np.arange(n) // 64) % 64 < 32, np.uint64(0), np.uint64(2**64 - 1))
    else:
        a0 = inputs.heavy_duplicates_u64(n, 19) * np.uint64(2**60)
    a = a0.copy()
    t, levels = orc.smoothed_partition(a, P50, seed=5, b=64, gmax=64, smin=16, base=256)
    assert t == int((a0 <= np.uint64(P50)).sum())
    assert np.all(a[:t] <= np.uint64(P50)) and np.all(a[t:] > np.uint64(P50))
    assert np.array_equal(np.sort(a), np.sort(a0))
    assert levels >= 1


def test_strided_partition(orc):
    n = 100000
    a0 = inputs.uniform_u64(n, 27)
    a = a0.copy()
    t = orc.strided_partition(a, P50, 16, 32)
    assert t == int((a0 <= np.uint64(P50)).sum())
    assert np.all(a[:t] <= np.uint64(P50)) and np.all(a[t:] > np.uint64(P50))
    assert np.array_equal(np.sort(a), np.sort(a0))


def test_determinism(orc):
    a0 = inputs.uniform_u64(50000, 2)
    a1, a2 = a0.copy(), a0.copy()
    orc.smoothed_partition(a1, P50, seed=9)
    orc.smoothed_partition(a2, P50, seed=9)
    assert np.array_equal(a1, a2)
