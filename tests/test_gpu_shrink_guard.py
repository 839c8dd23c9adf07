"""GPU parity of the residual-shrink guard of LP_SMOOTHED.

When the recursion of Sec. 4 keeps a range open at the level cap (or fails to
shrink it twice), the range goes to the Blocked-Prefix-Sum partition of Sec. 3
(the Hybrid scheme of Theorem 4.3).  lp_ctx_set_level_cap lowers the cap so a
test reaches that path on purpose.  The input is adversarial for one step:
each whole line is predecessors or successors, so each group's predecessor
fraction varies by whole lines and level 0 leaves a wide open range, more
than all CTAs hold on chip.  Whichever path finishes it, the
split must equal the oracle's and each side must hold the oracle's side as a
multiset.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2004_12532_gb300 import binding as lp
from paper_2004_12532_gb300 import inputs
from tests.gpu_util import check_partition, to_dev, to_host

pytestmark = pytest.mark.gpu

HANDOFF = (1 << 64) - 1  # the level record's g of a handed-over range


@pytest.fixture(scope="module")
def ctx():
    from paper_2004_12532_gb300 import build
    build.build()
    c = lp.Ctx(0)
    yield c
    c.set_level_cap(0)
    c.close()


def line_coins(n, line_keys, seed, bits=64):
    """Lines of line_keys keys, each line independently all small keys or all
    large keys (a fair seeded coin per line), the keys themselves seeded
    uniform within their half of the key range.  A group's predecessor count
    is then a sum of independent whole lines, the widest spread Prop. 4.2
    allows: one step leaves about 28% of the array open."""
    u = inputs.uniform_u64(n, seed) if bits == 64 else inputs.uniform_u32(n, seed)
    half = u.dtype.type(1 << (bits - 1))
    lines = -(-n // line_keys)
    coin = (inputs.uniform_u64(lines, seed ^ 0x77) >> np.uint64(63)) == 0
    low = np.repeat(coin, line_keys)[:n]
    return np.where(low, u % half, u | half).astype(u.dtype)


def levels_of(ctx):
    return [(lo, hi, g) for lo, hi, _, g, _ in ctx.level_stats() if hi > lo]


@pytest.mark.parametrize("cap", [1, 2, 0])
def test_handoff_u64(ctx, cap):
    n = (1 << 25) + 3
    host = line_coins(n, 256, 0x5A1)
    pivot = inputs.quantile_pivot(1, 2)
    ctx.set_level_cap(cap)
    dev = to_dev(host)
    t = lp.lp_partition_u64(ctx, dev, pivot, lp.LP_SMOOTHED, seed=3)
    lv = levels_of(ctx)
    ctx.set_level_cap(0)
    out = to_host(dev, np.uint64)
    ref = host.copy()
    check_partition(out, host, t, oracle.partition(ref, pivot), pivot)
    gs = [g for _, _, g in lv]
    if cap == 1:  # level 0 leaves more than the CTAs hold: handed over at level 1
        assert len(lv) >= 2 and gs[1] == HANDOFF, lv
    if HANDOFF in gs:  # the handoff ends the recursion
        assert gs.index(HANDOFF) == len(gs) - 1
        assert cap == 0 or gs.index(HANDOFF) <= cap


def test_handoff_u32(ctx):
    n = (1 << 26) + 7
    host = line_coins(n, 512, 0x5A2, bits=32)
    pivot = inputs.quantile_pivot(1, 2, 32)
    ctx.set_level_cap(1)
    dev = to_dev(host)
    t = lp.lp_partition_u32(ctx, dev, pivot, lp.LP_SMOOTHED, seed=4)
    gs = [g for _, _, g in levels_of(ctx)]
    ctx.set_level_cap(0)
    out = to_host(dev, np.uint32)
    ref = host.copy()
    check_partition(out, host, t, oracle.partition(ref, pivot), pivot)
    assert gs[1] == HANDOFF, gs


def test_handoff_kv(ctx):
    n = (1 << 24) + 5
    keys = line_coins(n, 256, 0x5A3)
    vals = np.arange(n, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)
    pivot = inputs.quantile_pivot(1, 2)
    ctx.set_level_cap(1)
    dk, dv = to_dev(keys), to_dev(vals)
    t = lp.lp_partition_kv_u64(ctx, dk, dv, pivot, lp.LP_SMOOTHED, seed=5)
    gs = [g for _, _, g in levels_of(ctx)]
    ctx.set_level_cap(0)
    ok, ov = to_host(dk, np.uint64), to_host(dv, np.uint64)
    rk, rv = keys.copy(), vals.copy()
    t_ref = oracle.partition_kv(rk, rv, pivot)
    assert t == t_ref and gs[1] == HANDOFF, (t, t_ref, gs)
    # each side's (key, payload) pairs as a multiset
    for sl in (slice(0, t), slice(t, n)):
        a = np.lexsort((ov[sl], ok[sl]))
        b = np.lexsort((rv[sl], rk[sl]))
        assert np.array_equal(ok[sl][a], rk[sl][b]) and np.array_equal(ov[sl][a], rv[sl][b])


def test_async_split_and_cap_bounds(ctx):
    """The async form gives the same split; caps at or above LP_MAX_LEVELS are
    refused."""
    n = (1 << 25) + 1
    host = line_coins(n, 256, 0x5A4)
    pivot = inputs.quantile_pivot(1, 2)
    ctx.set_level_cap(1)
    dev = to_dev(host)
    d = torch.zeros(1, dtype=torch.int64, device="cuda")
    lp.lp_partition_u64_async(ctx, dev, pivot, d, lp.LP_SMOOTHED, seed=6)
    ctx.wait()
    ctx.set_level_cap(0)
    assert int(d.item()) == oracle.count(host, pivot)
    with pytest.raises(lp.LPError):
        ctx.set_level_cap(lp.LP_MAX_LEVELS)
