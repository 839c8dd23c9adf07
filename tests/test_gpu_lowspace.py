"""GPU parity of the Blocked-Prefix-Sum (low-space) partition and of the
variants that clean up with it (Strided, Hybrid), against the serial oracle:
exact split and exact multiset of each side.

Small block sizes force many MakeSuccessorHeavy and Reorder levels at sizes the
oracle checks in seconds; both role-swap paths (predecessors the minority and
the majority) and the paper's base case (innermost prefix at most 5B) are
covered, as are the full-size-style default parameters (B = 4096).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2004_12532_gb300 import binding as lp
from paper_2004_12532_gb300 import inputs
from tests.gpu_util import check_partition, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2004_12532_gb300 import build
    build.build()
    c = lp.Ctx(0)
    yield c
    c.close()


@pytest.mark.parametrize("n", [1, 2, 3, 100, 5000, 65536 + 3, 1000003])
@pytest.mark.parametrize("B", [16, 64, 4096])
@pytest.mark.parametrize("q", [(1, 100), (1, 2), (7, 10), (99, 100)])
def test_lowspace_paper_base(ctx, n, B, q):
    host = inputs.uniform_u64(n, n * 7 + B)
    pv = inputs.quantile_pivot(*q)
    dev = to_dev(host)
    t = lp.lp_lowspace_partition(ctx, dev, pv, B=B, base_keys=0)
    check_partition(to_host(dev, np.uint64), host, t, oracle.count(host, pv), pv)


@pytest.mark.parametrize("n", [(1 << 22) + 17, (1 << 23) + 5])
@pytest.mark.parametrize("q", [(1, 2), (4, 5)])
def test_lowspace_on_chip_base(ctx, n, q):
    host = inputs.uniform_u64(n, n + q[0])
    pv = inputs.quantile_pivot(*q)
    dev = to_dev(host)
    t = lp.lp_lowspace_partition(ctx, dev, pv, B=4096, base_keys=1 << 20)
    check_partition(to_host(dev, np.uint64), host, t, oracle.count(host, pv), pv)


@pytest.mark.parametrize("n", [5000, (1 << 21) + 9])
def test_lowspace_u32(ctx, n):
    host = inputs.uniform_u32(n, n)
    pv = inputs.quantile_pivot(2, 3, 32)
    dev = to_dev(host)
    t = lp.lp_lowspace_partition(ctx, dev, pv, B=64)
    check_partition(to_host(dev, np.uint32), host, t, oracle.count(host, pv), pv)


@pytest.mark.parametrize("variant", [lp.LP_LOWSPACE, lp.LP_STRIDED, lp.LP_HYBRID])
@pytest.mark.parametrize("n,offset", [(9000, 0), ((1 << 22) + 37, 1), ((1 << 23) + 1, 0)])
def test_variants_u64(ctx, variant, n, offset):
    host = inputs.uniform_u64(n, n + variant)
    pv = inputs.quantile_pivot(3, 5)
    buf = to_dev(np.concatenate([np.zeros(offset, np.uint64), host]))
    view = buf[offset:]
    t = lp.lp_partition_u64(ctx, view, pv, variant, seed=3)
    check_partition(to_host(view, np.uint64), host, t, oracle.count(host, pv), pv)


@pytest.mark.parametrize("variant", [lp.LP_LOWSPACE, lp.LP_STRIDED, lp.LP_HYBRID])
def test_variants_u32_kv(ctx, variant):
    n = (1 << 22) + 3
    h32 = inputs.uniform_u32(n, 5)
    pv32 = inputs.quantile_pivot(1, 2, 32)
    d32 = to_dev(h32)
    t = lp.lp_partition_u32(ctx, d32, pv32, variant, seed=1)
    check_partition(to_host(d32, np.uint32), h32, t, oracle.count(h32, pv32), pv32)
    keys = inputs.uniform_u64(n, 6)
    vals = np.arange(n, dtype=np.uint64)
    pv = inputs.quantile_pivot(1, 3)
    dk, dv = to_dev(keys), to_dev(vals)
    t = lp.lp_partition_kv_u64(ctx, dk, dv, pv, variant, seed=2)
    ko, vo = to_host(dk, np.uint64), to_host(dv, np.uint64)
    check_partition(ko, keys, t, oracle.count(keys, pv), pv)
    assert np.array_equal(keys[vo.astype(np.int64)], ko)


def test_strided_adversarial_period(ctx):
    """Input aligned with the strides: the Strided step leaves a wide open
    range, which the low-space cleanup must still finish."""
    n = 1 << 22
    host = np.where((np.arange(n) // 128) % 2432 < 1216, np.uint64(1), np.uint64(2**64 - 1))
    dev = to_dev(host)
    t = lp.lp_partition_u64(ctx, dev, 5, lp.LP_STRIDED)
    check_partition(to_host(dev, np.uint64), host, t, oracle.count(host, 5), 5)


@pytest.mark.parametrize("variant", [lp.LP_LOWSPACE, lp.LP_STRIDED, lp.LP_HYBRID])
@pytest.mark.parametrize("frac", [(1, 3), (1, 2), (7, 10)])
def test_variants_kv_repeated(ctx, variant, frac):
    """Key + payload through the low-space kernel with the predecessors the
    minority, about half, and the majority (the reversed view), 12 seeded
    inputs each: a fault that depends on timing between CTAs (two warps
    writing one shared-memory word) shows up as duplicated key/payload pairs."""
    pv = inputs.quantile_pivot(*frac)
    flip = torch.tensor(-(1 << 63), dtype=torch.int64, device="cuda")
    p_signed = pv - (1 << 63)
    for r in range(12):
        n = (1 << 22) + 3 + 1000 * r
        keys = torch.empty(n, dtype=torch.int64, device="cuda")
        lp.lp_fill_uniform_u64(keys, 7000 + 31 * r + variant)
        kin = keys.clone()
        vals = torch.arange(n, dtype=torch.int64, device="cuda")
        t = lp.lp_partition_kv_u64(ctx, keys, vals, pv, variant, seed=r)
        ki, ko = kin ^ flip, keys ^ flip  # signed order of the flipped bits = unsigned order
        assert t == int((ki <= p_signed).sum())
        assert int((ko[:t] > p_signed).sum()) == 0 and int((ko[t:] <= p_signed).sum()) == 0
        assert torch.equal(torch.sort(kin)[0], torch.sort(keys)[0])  # a permutation
        assert torch.equal(kin[vals], keys)  # every payload still names its key


def structured_u64(kind, n, seed):
    """Inputs whose blocks hold no predecessors, only predecessors, or runs of
    either: the Reorder's per-block target ranges are then empty, full, or
    cut at block edges."""
    rng = np.random.default_rng(seed)
    u = inputs.uniform_u64(n, seed)
    if kind == "sorted":
        return np.sort(u)
    if kind == "reverse":
        return np.sort(u)[::-1].copy()
    if kind == "equal":
        return np.full(n, np.uint64(1 << 62), dtype=np.uint64)
    if kind == "block_runs":  # runs of 4096 keys alternately below and above 2^63
        lo = u >> np.uint64(1)
        hi = lo | np.uint64(1 << 63)
        run = (np.arange(n) // 4096) % 2 == 0
        return np.where(run, lo, hi)
    if kind == "ragged_runs":  # runs of random lengths alternately below and above 2^63
        lens = rng.integers(1, 9000, size=n // 1000 + 2)
        side = np.repeat(np.arange(lens.size) % 2 == 0, lens)[:n]
        lo = u >> np.uint64(1)
        return np.where(side, lo, lo | np.uint64(1 << 63))
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["sorted", "reverse", "equal", "block_runs", "ragged_runs"])
@pytest.mark.parametrize("q", [(1, 100), (1, 2), (99, 100)])
def test_lowspace_structured(ctx, kind, q):
    """Default parameters (B = 4096, the innermost prefix on chip) on
    (1 << 23) + 11 keys: several Reorder levels, blocks with no targets and
    blocks whose targets fill several rounds; split and both sides' multisets
    against the oracle."""
    n = (1 << 23) + 11
    host = structured_u64(kind, n, 41 + q[0])
    pv = inputs.quantile_pivot(*q) if kind != "equal" else (1 << 62) - (q[0] == 1)
    dev = to_dev(host)
    t = lp.lp_partition_u64(ctx, dev, pv, lp.LP_LOWSPACE)
    check_partition(to_host(dev, np.uint64), host, t, oracle.count(host, pv), pv)
