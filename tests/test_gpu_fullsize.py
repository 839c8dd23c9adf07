"""Parity at the workloads' full sizes, in the launch configuration bench.py
times (one cooperative launch over the whole array), checked by properties
that hold at any size, computed on the device:

  * the split equals the number of keys <= pivot in the input;
  * every key left of the split is <= pivot, every key right of it > pivot;
  * each side is a permutation of the input's keys of that side (sorted
    copies are equal), so the output permutes the input; and
    for key + payload, every output key equals the input key at its payload
    (payload = original index), so pairs moved together.

Sizes: 2^30 uint64 at the 1%, 50% and 99% quantile pivots (8 GiB), 2^31
uint32 (8 GiB), 2^29 key + payload pairs, the Strided / low-space / Hybrid
variants and the low-space form with values kept in key order at 2^30, and
the 4096-instance batch (1.8 G keys).
"""
import numpy as np
import pytest
import torch

from paper_2004_12532_gb300 import binding as lp
from paper_2004_12532_gb300 import inputs
from tests.gpu_util import unsigned_key

pytestmark = pytest.mark.gpu

SIGN64 = -(1 << 63)
SIGN32 = -(1 << 31)


@pytest.fixture(scope="module")
def ctx():
    from paper_2004_12532_gb300 import build
    build.build()
    c = lp.Ctx(0)
    yield c
    c.close()


def signed_pivot(pivot, bits):
    """The signed value whose order among unsigned_key() matches pivot's."""
    v = pivot ^ (1 << (bits - 1))
    return v - (1 << bits) if v >= 1 << (bits - 1) else v


def check_props(inp, out, t, pivot, bits):
    ki, ko = unsigned_key(inp), unsigned_key(out)
    sp = signed_pivot(pivot, bits)
    assert t == int((ki <= sp).sum().item())
    assert bool((ko[:t] <= sp).all().item())
    assert bool((ko[t:] > sp).all().item())
    # per side (each side stays under torch.sort's 2^31 - 1 element limit)
    left = ki <= sp
    assert torch.equal(torch.sort(ki[left]).values, torch.sort(ko[:t]).values)
    del left
    assert torch.equal(torch.sort(ki[ki > sp]).values, torch.sort(ko[t:]).values)


@pytest.mark.parametrize("q", [1, 50, 99])
def test_u64_2pow30(ctx, q):
    n = 1 << 30
    pivot = inputs.quantile_pivot(q, 100, 64)
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    lp.lp_fill_uniform_u64(keys, 0xC0FF2 + q)
    inp = keys.clone()
    t = lp.lp_partition_u64(ctx, keys, pivot, seed=q)
    check_props(inp, keys, t, pivot, 64)


@pytest.mark.parametrize("variant", [lp.LP_STRIDED, lp.LP_LOWSPACE, lp.LP_HYBRID])
@pytest.mark.parametrize("q", [(1, 2), (99, 100)])
def test_variants_u64_2pow30(ctx, variant, q):
    n = 1 << 30
    pivot = inputs.quantile_pivot(q[0], q[1], 64)
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    lp.lp_fill_uniform_u64(keys, 0xC0FF3 + variant)
    inp = keys.clone()
    t = lp.lp_partition_u64(ctx, keys, pivot, variant=variant, seed=3)
    check_props(inp, keys, t, pivot, 64)
    assert ctx.aux_bytes <= 0.01 * n * 8


def test_u32_2pow31(ctx):
    n = 1 << 31
    pivot = inputs.quantile_pivot(1, 2, 32)
    keys = torch.empty(n, dtype=torch.int32, device="cuda")
    lp.lp_fill_uniform_u32(keys, 0xC0FF4)
    inp = keys.clone()
    t = lp.lp_partition_u32(ctx, keys, pivot, seed=5)
    check_props(inp, keys, t, pivot, 32)


def test_kv_2pow29(ctx):
    n = 1 << 29
    pivot = inputs.quantile_pivot(1, 2, 64)
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    vals = torch.empty(n, dtype=torch.int64, device="cuda")
    lp.lp_fill_uniform_u64(keys, 0xC0FF5)
    lp.lp_fill_iota_u64(vals)
    inp = keys.clone()
    t = lp.lp_partition_kv_u64(ctx, keys, vals, pivot, seed=7)
    ko = unsigned_key(keys)
    sp = signed_pivot(pivot, 64)
    assert t == int((unsigned_key(inp) <= sp).sum().item())
    assert bool((ko[:t] <= sp).all().item()) and bool((ko[t:] > sp).all().item())
    # every pair moved together, and every original index appears once
    assert torch.equal(keys, inp[vals])
    assert torch.equal(torch.sort(vals).values, torch.arange(n, device="cuda"))


def test_batched_4096_instances(ctx):
    count = 4096
    sizes = inputs.log_uniform_sizes(count, 0xC0FF2, 8, 22)
    offs, tot = [], 0
    for m in sizes:
        offs.append(tot)
        tot += (int(m) + 1) & ~1
    buf = torch.empty(tot, dtype=torch.int64, device="cuda")
    lp.lp_fill_uniform_u64(buf, 0xC0FF6)
    rng = np.random.default_rng(0xC0FF2)
    pick = [o + int(rng.integers(0, m)) for o, m in zip(offs, sizes)]
    pv = buf[torch.tensor(pick, device="cuda")].cpu().numpy()
    pivots = [int(x) & 0xFFFFFFFFFFFFFFFF for x in pv]
    inp = buf.clone()
    views = [buf[o:o + int(m)] for o, m in zip(offs, sizes)]
    splits = torch.zeros(count, dtype=torch.int64, device="cuda")
    b = lp.Batch(ctx, views, pivots, splits, seed=1)
    b.launch()
    b.wait()
    b.close()
    # checked in groups of segments of about 2^27 keys (bounded memory): per
    # element its segment, its place in the segment, its segment's pivot
    spv = [signed_pivot(p, 64) for p in pivots]
    s0 = 0
    while s0 < count:
        s1, keys_in_group = s0, 0
        while s1 < count and (keys_in_group == 0 or keys_in_group + int(sizes[s1]) <= 1 << 27):
            keys_in_group += int(sizes[s1])
            s1 += 1
        g = s1 - s0
        seg_len = torch.tensor([int(m) for m in sizes[s0:s1]], device="cuda")
        seg_off = torch.tensor(offs[s0:s1], device="cuda")
        seg_id = torch.repeat_interleave(torch.arange(g, device="cuda"), seg_len)
        starts = torch.cumsum(seg_len, 0) - seg_len
        pos = torch.arange(keys_in_group, device="cuda") - starts[seg_id]
        idx = seg_off[seg_id] + pos
        sp = torch.tensor(spv[s0:s1], device="cuda")[seg_id]
        ki, ko = unsigned_key(inp[idx]), unsigned_key(buf[idx])
        counts = torch.zeros(g, dtype=torch.int64, device="cuda").index_add_(
            0, seg_id, (ki <= sp).to(torch.int64))
        assert torch.equal(counts, splits[s0:s1])
        assert bool(((pos < splits[s0:s1][seg_id]) == (ko <= sp)).all().item())
        # each segment is a permutation of its input: sort by (segment, key)
        def seg_sorted(k):
            order = torch.argsort(k, stable=True)
            order = order[torch.argsort(seg_id[order], stable=True)]
            return k[order]
        assert torch.equal(seg_sorted(ki), seg_sorted(ko))
        s0 = s1


@pytest.mark.parametrize("q", [50, 99])
def test_implicit_u64_2pow30(ctx, q):
    """The fully in-place form (block values kept in key order), 2^30 keys,
    at the half and the 99% (role-swapped) pivots."""
    n = 1 << 30
    pivot = inputs.quantile_pivot(q, 100, 64)
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    lp.lp_fill_uniform_u64(keys, 0xC0FF6 + q)
    inp = keys.clone()
    t = lp.lp_lowspace_implicit_partition(ctx, keys, pivot)
    check_props(inp, keys, t, pivot, 64)


def test_host_array_u64_2pow30(ctx):
    """The host-array entry point at the full size: a pinned 8 GiB array,
    partitioned in place through lp_partition_host_u64, checked on the
    device."""
    n = 1 << 30
    pivot = inputs.quantile_pivot(1, 2, 64)
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    lp.lp_fill_uniform_u64(keys, 0xC0FF7)
    host = torch.empty(n, dtype=torch.int64, pin_memory=True)
    host.copy_(keys)
    t = lp.lp_partition_host(ctx, host, pivot, seed=1)
    out = host.to("cuda")
    check_props(keys, out, t, pivot, 64)
