"""GPU parity: the CUDA Smoothed Striding path (through the C ABI) against the
serial CPU oracle, bit-exact on the split and on the multiset of each side.

Sizes span several lines, groups and chunks with ragged tails, unaligned base
pointers, the small single-CTA path and its boundary, skewed pivots and
adversarial patterns.  The single-step tests pin the hot kernel to the
paper's Partial Partition Step exactly (same X, same v_min / v_max / count,
each group a predecessors-first permutation of itself).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2004_12532_gb300 import binding as lp
from paper_2004_12532_gb300 import inputs
from tests.gpu_util import check_partition, to_dev, to_host

pytestmark = pytest.mark.gpu

P50 = inputs.quantile_pivot(1, 2)


@pytest.fixture(scope="module")
def ctx():
    from paper_2004_12532_gb300 import build
    build.build()
    c = lp.Ctx(0)
    yield c
    c.close()


def run_u64(ctx, host, pivot, seed=1, variant=lp.LP_SMOOTHED, offset=0):
    buf = to_dev(np.concatenate([np.zeros(offset, np.uint64), host]))
    view = buf[offset:]
    t = lp.lp_partition_u64(ctx, view, pivot, variant, seed)
    torch.cuda.synchronize()
    out = to_host(view, np.uint64)
    return t, out


# ------------------------------------------------------------ single step
def group_of_positions(n, b, g, X):
    L = -(-n // b)
    lines = np.arange(L, dtype=np.int64)
    grp = (lines % g - X[lines // g].astype(np.int64)) % g
    return np.repeat(grp, b)[:n]


@pytest.mark.parametrize("n,b,g,strided", [
    (1 << 16, 64, 16, 0), (1 << 16, 64, 16, 1), (100000, 32, 37, 0),
    (1 << 20, 64, 304, 0), ((1 << 20) + 4096 + 2, 64, 100, 0), (4096, 8, 3, 0),
    (2 * 1000, 2, 7, 0), (5000, 64, 3, 0), (30000, 16, 1, 0), (1 << 20, 64, 3000, 0),
    ((1 << 22) + 18, 32, 2000, 0), (1 << 21, 64, 1, 0), (1 << 22, 64, 2432, 1),
    ((1 << 22) + 6, 128, 777, 0), (1 << 21, 128, 5000, 0)])
def test_step_parity(ctx, n, b, g, strided):
    """One Partial Partition Step: v_min, v_max and the count equal the
    oracle's for the same X; every group is a predecessors-first permutation
    of its own slots; A[p] <= pivot below v_min and > pivot from v_max."""
    host = inputs.uniform_u64(n, n + g)
    seed, level = 77, 2
    dev = to_dev(host)
    vmin, vmax, cnt = lp.lp_smoothed_step(ctx, dev, P50, b, g, seed, level, bool(strided))
    out = to_host(dev, np.uint64)
    s = oracle.num_chunks(n, b, g)
    X = np.zeros(s, np.uint64) if strided else oracle.draw_X(seed, level, s, g)
    ref = host.copy()
    _, _, rmin, rmax = oracle.smoothed_step(ref, P50, b, g, X)
    assert (vmin, vmax) == (rmin, rmax)
    assert cnt == oracle.count(host, P50)
    p = np.uint64(P50)
    assert np.all(out[:vmin] <= p) and np.all(out[vmax:] > p)
    grp = group_of_positions(n, b, g, X)
    order = np.lexsort((np.arange(n), grp))  # group-major, positions ascending
    g_sorted = grp[order]
    # per-group multiset: sort (group, key) pairs of input and output
    kin = np.lexsort((host[order], g_sorted))
    kout = np.lexsort((out[order], g_sorted))
    assert np.array_equal(host[order][kin], out[order][kout])
    # predecessors first inside every group, in group slot order
    flag = (out[order] <= p).astype(np.int8)
    same = g_sorted[1:] == g_sorted[:-1]
    assert not np.any(same & (flag[1:] > flag[:-1]))


def test_step_u32(ctx):
    n, b, g = 1 << 18, 128, 50
    host = inputs.uniform_u32(n, 5)
    pv = inputs.quantile_pivot(1, 3, 32)
    dev = to_dev(host)
    vmin, vmax, cnt = lp.lp_smoothed_step(ctx, dev, pv, b, g, 3, 0)
    ref = host.copy()
    X = oracle.draw_X(3, 0, oracle.num_chunks(n, b, g), g)
    _, _, rmin, rmax = oracle.smoothed_step(ref, pv, b, g, X)
    assert (vmin, vmax, cnt) == (rmin, rmax, oracle.count(host, pv))
    out = to_host(dev, np.uint32)
    assert np.array_equal(np.sort(out), np.sort(host))


def test_step_rejects_bad_args(ctx):
    dev = to_dev(inputs.uniform_u64(1000, 1))
    with pytest.raises(lp.LPError) as e:
        lp.lp_smoothed_step(ctx, dev[1:], P50, 8, 4)  # 8-byte offset: not 16-aligned
    assert e.value.status == lp.LP_ERR_MISALIGNED
    with pytest.raises(lp.LPError) as e:
        lp.lp_smoothed_step(ctx, dev, P50, 3, 4)  # 24-byte line
    assert e.value.status == lp.LP_ERR_INVALID_ARG
    with pytest.raises(lp.LPError) as e:
        lp.lp_smoothed_step(ctx, dev, P50, 512, 4)  # 4096-byte line: above the limit
    assert e.value.status == lp.LP_ERR_INVALID_ARG


# ------------------------------------------------------------ full partition
SIZES = [0, 1, 2, 3, 17, 255, 4095, 8191, 8192, 8193, 8194, 12345, 65536 + 7,
         (1 << 18) + 1, 1000003, (1 << 20), (1 << 22) + 37]


@pytest.mark.parametrize("n", SIZES)
def test_partition_u64_sizes(ctx, n):
    host = inputs.uniform_u64(n, 1000 + n)
    t, out = run_u64(ctx, host, P50, seed=n)
    check_partition(out, host, t, oracle.count(host, P50), P50)


@pytest.mark.parametrize("offset", [1, 2, 3])
@pytest.mark.parametrize("n", [9000, 300001, (1 << 20) + 5])
def test_partition_u64_unaligned(ctx, n, offset):
    host = inputs.uniform_u64(n, 7 * n + offset)
    t, out = run_u64(ctx, host, P50, offset=offset)
    check_partition(out, host, t, oracle.count(host, P50), P50)


@pytest.mark.parametrize("q", [(1, 100), (1, 2), (99, 100)])
def test_partition_u64_quantiles(ctx, q):
    n = (1 << 22) + 1234
    pv = inputs.quantile_pivot(*q)
    host = inputs.uniform_u64(n, 31)
    t, out = run_u64(ctx, host, pv)
    check_partition(out, host, t, oracle.count(host, pv), pv)


@pytest.mark.parametrize("pivot", [0, 2**64 - 1, 5])
def test_partition_u64_extreme_pivots(ctx, pivot):
    n = 500000
    host = inputs.uniform_u64(n, 3)
    host[::1000] = 5
    t, out = run_u64(ctx, host, pivot)
    check_partition(out, host, t, oracle.count(host, pivot), pivot)


@pytest.mark.parametrize("kind", ["sorted", "reverse", "equal", "dup16", "period", "lines"])
def test_partition_u64_patterns(ctx, kind):
    n = (1 << 21) + 99
    if kind == "sorted":
        host = inputs.sorted_u64(n, 4)
    elif kind == "reverse":
        host = inputs.reverse_sorted_u64(n, 4)
    elif kind == "equal":
        host = np.full(n, P50, dtype=np.uint64)
    elif kind == "dup16":
        host = inputs.heavy_duplicates_u64(n, 4) << np.uint64(60)
    elif kind == "period":
        host = np.where((np.arange(n) // 512) % 304 < 152, np.uint64(1), np.uint64(2**64 - 1))
    else:
        host = np.where((np.arange(n) // 4096) % 2 == 0, np.uint64(0), np.uint64(2**64 - 1))
    t, out = run_u64(ctx, host, P50)
    check_partition(out, host, t, oracle.count(host, P50), P50)


@pytest.mark.parametrize("variant", [lp.LP_STRIDED])
def test_partition_strided(ctx, variant):
    n = (1 << 22) + 3
    host = inputs.uniform_u64(n, 8)
    t, out = run_u64(ctx, host, P50, variant=variant)
    check_partition(out, host, t, oracle.count(host, P50), P50)


@pytest.mark.parametrize("n", [5, 16383, 16384, 16385, (1 << 20) + 3, (1 << 23) + 1])
@pytest.mark.parametrize("offset", [0, 1, 3])
def test_partition_u32(ctx, n, offset):
    host = inputs.uniform_u32(n, n + offset)
    pv = inputs.quantile_pivot(1, 2, 32)
    buf = to_dev(np.concatenate([np.zeros(offset, np.uint32), host]))
    view = buf[offset:]
    t = lp.lp_partition_u32(ctx, view, pv)
    out = to_host(view, np.uint32)
    check_partition(out, host, t, oracle.count(host, pv), pv)


@pytest.mark.parametrize("kind", ["uniform_q1", "uniform_q99", "sorted", "reverse", "equal",
                                  "dup16", "period", "lines"])
def test_partition_u32_patterns(ctx, kind):
    """The 16-slot line swap of 4-byte keys on inputs that make one side's
    wrong keys all move or only a prefix of them (every lane, or one), with
    lines that are pure from the start and lines that are all wrong."""
    n = (1 << 22) + 77
    pv = inputs.quantile_pivot(1, 2, 32)
    u = inputs.uniform_u32(n, 11)
    if kind == "uniform_q1":
        host, pv = u, inputs.quantile_pivot(1, 100, 32)
    elif kind == "uniform_q99":
        host, pv = u, inputs.quantile_pivot(99, 100, 32)
    elif kind == "sorted":
        host = np.sort(u)
    elif kind == "reverse":
        host = np.sort(u)[::-1].copy()
    elif kind == "equal":
        host = np.full(n, np.uint32(pv), dtype=np.uint32)
    elif kind == "dup16":
        host = (u & np.uint32(15)) << np.uint32(28)
    elif kind == "period":
        host = np.where((np.arange(n) // 1024) % 304 < 152, np.uint32(1), np.uint32(2**32 - 1))
    else:
        host = np.where((np.arange(n) // 512) % 2 == 0, np.uint32(0), np.uint32(2**32 - 1))
    dev = to_dev(host)
    t = lp.lp_partition_u32(ctx, dev, pv)
    check_partition(to_host(dev, np.uint32), host, t, oracle.count(host, pv), pv)


@pytest.mark.parametrize("n", [100, 4096, 4097, 300007, (1 << 21) + 11])
@pytest.mark.parametrize("offset", [0, 1])
def test_partition_kv(ctx, n, offset):
    keys = inputs.uniform_u64(n, 55 + n)
    vals = np.arange(n, dtype=np.uint64)
    pv = inputs.quantile_pivot(2, 5)
    kb = to_dev(np.concatenate([np.zeros(offset, np.uint64), keys]))
    vb = to_dev(np.concatenate([np.zeros(offset, np.uint64), vals]))
    t = lp.lp_partition_kv_u64(ctx, kb[offset:], vb[offset:], pv)
    ko = to_host(kb[offset:], np.uint64)
    vo = to_host(vb[offset:], np.uint64)
    check_partition(ko, keys, t, oracle.count(keys, pv), pv)
    # the payload still names its key: keys_in[vals_out] == keys_out
    assert np.array_equal(keys[vo.astype(np.int64)], ko)
    assert np.array_equal(np.sort(vo), vals)


def test_async_split_and_determinism(ctx):
    n = (1 << 21) + 5
    host = inputs.uniform_u64(n, 9)
    a = to_dev(host)
    b = to_dev(host)
    sa = torch.zeros(1, dtype=torch.int64, device="cuda")
    sb = torch.zeros(1, dtype=torch.int64, device="cuda")
    lp.lp_partition_u64_async(ctx, a, P50, sa, seed=4)
    lp.lp_partition_u64_async(ctx, b, P50, sb, seed=4)
    torch.cuda.synchronize()
    assert int(sa.item()) == int(sb.item()) == oracle.count(host, P50)
    assert torch.equal(a, b)  # same input and seed: same bytes


def test_invalid_arguments(ctx):
    with pytest.raises(lp.LPError) as e:
        lp.lib()  # loaded
        import ctypes
        t = ctypes.c_uint64()
        ctx.check(lp.lib().lp_partition_u64(ctx.h, None, 10, 0, 0, 0, None, ctypes.byref(t)))
    assert e.value.status == lp.LP_ERR_INVALID_ARG
    empty = torch.zeros(0, dtype=torch.int64, device="cuda")
    assert lp.lp_partition_u64(ctx, empty, 5) == 0
