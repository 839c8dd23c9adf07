"""GPU parity of the Blocked-Prefix-Sum partition with the block values kept
in the order of each block's keys (Sec. 3, Lemma bitstore2).

- The first three phases (count and role swap, MakeSuccessorHeavy, the
  prefix phase with its pair reordering and encodings) are compared with the
  oracle's element by element: the whole array must be bit-identical.
- The whole partition: the oracle's split, each side the same multiset.
Inputs: uniform keys (unequal pairs: the order encoding), keys mod 2 and mod 5
(mostly equal pairs: the overwrite encoding), sorted keys; pivots from 1% to
99% (both roles); block sizes from the paper's minimum 4 ceil(log2(n+1)) + 2
to 4096; sizes that leave a ragged last block.
"""
import numpy as np
import pytest

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


def _input(n, kind, seed, q, bits=64):
    a = inputs.uniform_u64(n, seed) if bits == 64 else inputs.uniform_u32(n, seed)
    pv = inputs.quantile_pivot(*q, bits)
    if kind == "mod2":
        a = a % a.dtype.type(2)
        pv = 0
    elif kind == "mod5":
        a = a % a.dtype.type(5)
        pv = q[0] * 5 // q[1]
    elif kind == "sorted":
        a = np.sort(a)
    return a, pv


def _bmin(n):
    return 4 * oracle.bits_for(n) + 2


@pytest.mark.parametrize("n", [2, 3, 200, 5000, 65536 + 3, 1000003, (1 << 22) + 17])
@pytest.mark.parametrize("kind", ["uniform", "mod2", "mod5", "sorted"])
@pytest.mark.parametrize("q", [(1, 100), (1, 2), (7, 10)])
@pytest.mark.parametrize("B", [0, 256, 4096])
def test_prefix_phase_bit_exact_u64(ctx, n, kind, q, B):
    a, pv = _input(n, kind, 11 * n + q[0], q)
    Beff = B or _bmin(n)
    if Beff < _bmin(n):
        pytest.skip("block below the encoding size")
    dev = to_dev(a)
    t = lp.lp_lowspace_implicit_prefix(ctx, dev, pv, B=B)
    ref = a.copy()
    t_ref, _ = oracle.implicit_prefix(ref, pv, Beff)
    assert t == t_ref
    out = to_host(dev, np.uint64)
    bad = np.nonzero(out != ref)[0]
    assert bad.size == 0, (bad[:8], out[bad[:8]], ref[bad[:8]])


@pytest.mark.parametrize("n", [5000, 1000003])
@pytest.mark.parametrize("kind", ["uniform", "mod2"])
@pytest.mark.parametrize("q", [(1, 3), (4, 5)])
def test_prefix_phase_bit_exact_u32(ctx, n, kind, q):
    a, pv = _input(n, kind, 5 * n + q[0], q, bits=32)
    B = 128
    dev = to_dev(a)
    t = lp.lp_lowspace_implicit_prefix(ctx, dev, pv, B=B)
    ref = a.astype(np.uint64)  # the oracle's steps commute with widening
    t_ref, _ = oracle.implicit_prefix(ref, pv, B)
    assert t == t_ref
    assert np.array_equal(to_host(dev, np.uint32), ref.astype(np.uint32))


@pytest.mark.parametrize("n", [1, 2, 3, 200, 5000, 65536 + 3, 1000003, (1 << 22) + 17])
@pytest.mark.parametrize("kind", ["uniform", "mod2", "mod5", "sorted"])
@pytest.mark.parametrize("q", [(1, 100), (1, 2), (99, 100)])
def test_partition_u64(ctx, n, kind, q):
    a, pv = _input(n, kind, 3 * n + q[1], q)
    dev = to_dev(a)
    t = lp.lp_lowspace_implicit_partition(ctx, dev, pv, B=0 if n < 5000 else 4096,
                                          base_keys=0)
    check_partition(to_host(dev, np.uint64), a, t, oracle.count(a, pv), pv)


@pytest.mark.parametrize("n", [(1 << 22) + 17, (1 << 23) + 5])
@pytest.mark.parametrize("q", [(1, 2), (4, 5)])
@pytest.mark.parametrize("B", [0, 4096])
def test_partition_on_chip_base(ctx, n, q, B):
    a, pv = _input(n, "uniform", n + q[0], q)
    dev = to_dev(a)
    t = lp.lp_lowspace_implicit_partition(ctx, dev, pv, B=B, base_keys=1 << 20)
    check_partition(to_host(dev, np.uint64), a, t, oracle.count(a, pv), pv)


@pytest.mark.parametrize("n", [5000, (1 << 21) + 9])
@pytest.mark.parametrize("kind", ["uniform", "mod2"])
def test_partition_u32(ctx, n, kind):
    a, pv = _input(n, kind, n, (2, 3), bits=32)
    dev = to_dev(a)
    t = lp.lp_lowspace_implicit_partition(ctx, dev, pv, B=128)
    check_partition(to_host(dev, np.uint32), a, t, oracle.count(a, pv), pv)


def test_errors(ctx):
    import torch
    n = 100000
    keys = torch.zeros(n, dtype=torch.int64, device="cuda")
    with pytest.raises(lp.LPError):
        lp.lp_lowspace_implicit_partition(ctx, keys, 5, B=_bmin(n) - 1)
    empty = torch.zeros(0, dtype=torch.int64, device="cuda")
    assert lp.lp_lowspace_implicit_partition(ctx, empty, 5) == 0
    # the context still works after the refusal
    a, pv = _input(n, "uniform", 1, (1, 2))
    dev = to_dev(a)
    t = lp.lp_lowspace_implicit_partition(ctx, dev, pv, B=_bmin(n))
    check_partition(to_host(dev, np.uint64), a, t, oracle.count(a, pv), pv)
