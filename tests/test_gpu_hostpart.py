"""GPU parity of the host-array partition (lp_partition_host_*): a pinned or
pageable CPU array is partitioned in place through chunk uploads, device
partitions and copies back; compared with the oracle's split, the
postcondition and each side's multiset.  Sizes from empty to 16 chunks;
layouts that put all predecessors at one end or alternate by chunk-sized
blocks (the plan's hardest cases); both key widths; and the same result on
every run."""
import numpy as np
import pytest
import torch

import oracle
from paper_2004_12532_gb300 import binding as lp
from paper_2004_12532_gb300 import inputs
from tests.gpu_util import check_partition

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2004_12532_gb300 import build
    build.build()
    c = lp.Ctx(0)
    yield c
    c.close()


def _host(a, pinned=True):
    t = torch.from_numpy(a.view(np.int64 if a.dtype == np.uint64 else np.int32).copy())
    return t.pin_memory() if pinned else t


def _layout(a, kind):
    if kind == "sorted":
        return np.sort(a)
    if kind == "reverse":
        return np.sort(a)[::-1].copy()
    if kind == "blocks":  # chunk-sized runs alternating between the two sides
        n = a.size
        b = max(1, n // 7)
        s = np.sort(a)
        lo, hi = s[: n // 2], s[n // 2:]
        out = np.empty_like(a)
        i = j = k = 0
        while k < n:
            src = lo if (k // b) % 2 == 0 and i < lo.size or j >= hi.size else hi
            if src is lo:
                m = min(b - k % b, lo.size - i)
                out[k:k + m] = lo[i:i + m]
                i += m
            else:
                m = min(b - k % b, hi.size - j)
                out[k:k + m] = hi[j:j + m]
                j += m
            k += m
        return out
    return a


@pytest.mark.parametrize("n", [0, 1, 1000, (1 << 22) + 17, (1 << 23) + 5, (1 << 26) + 3])
@pytest.mark.parametrize("q", [(1, 100), (1, 2), (99, 100)])
def test_host_u64(ctx, n, q):
    a = inputs.uniform_u64(n, 2 * n + q[0])
    pv = inputs.quantile_pivot(*q)
    h = _host(a)
    t = lp.lp_partition_host(ctx, h, pv, seed=5)
    check_partition(h.numpy().view(np.uint64), a, t, oracle.count(a, pv), pv)


@pytest.mark.parametrize("kind", ["sorted", "reverse", "blocks"])
def test_host_layouts(ctx, kind):
    n = (1 << 25) + 11
    a = _layout(inputs.uniform_u64(n, 77), kind)
    pv = inputs.quantile_pivot(1, 2)
    h = _host(a)
    t = lp.lp_partition_host(ctx, h, pv)
    check_partition(h.numpy().view(np.uint64), a, t, oracle.count(a, pv), pv)


@pytest.mark.parametrize("n", [5000, (1 << 24) + 9])
def test_host_u32(ctx, n):
    a = inputs.uniform_u32(n, n)
    pv = inputs.quantile_pivot(2, 3, 32)
    h = _host(a)
    t = lp.lp_partition_host(ctx, h, pv)
    check_partition(h.numpy().view(np.uint32), a, t, oracle.count(a, pv), pv)


def test_host_pageable_and_repeatable(ctx):
    n = (1 << 24) + 3
    a = inputs.uniform_u64(n, 9)
    pv = inputs.quantile_pivot(3, 10)
    outs = []
    for pinned in (True, False, True):
        h = _host(a, pinned)
        t = lp.lp_partition_host(ctx, h, pv, seed=2)
        out = h.numpy().view(np.uint64).copy()
        check_partition(out, a, t, oracle.count(a, pv), pv)
        outs.append(out)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_host_errors(ctx):
    with pytest.raises(TypeError):
        lp.lp_partition_host(ctx, torch.zeros(4, dtype=torch.int64, device="cuda"), 1)
    h = torch.zeros(0, dtype=torch.int64)
    assert lp.lp_partition_host(ctx, h, 1) == 0
