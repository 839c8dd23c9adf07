"""GPU parity of the quicksort on the partition (Sec. 5, "A Full Quicksort").

The sorted array is unique, so the GPU result must equal the oracle's serial
quicksort byte for byte: uniform, sorted, reverse-sorted and heavy-duplicate
inputs (the four inputs of the n = 2^28 workload), uint64 and uint32, sizes
around the shared-memory cut (4096 keys), the one-CTA finish and several
partition levels, and views at odd 8-byte offsets.  At the workload's full
size the result is checked by properties: non-decreasing, and equal to a
library sort of the input.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2004_12532_gb300 import binding as lp
from paper_2004_12532_gb300 import inputs
from tests.gpu_util import to_dev, to_host, unsigned_key

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2004_12532_gb300 import build
    build.build()
    c = lp.Ctx(0)
    yield c
    c.close()


def make(kind, n, seed, dtype=np.uint64):
    if dtype == np.uint32:
        if kind == "uniform":
            return inputs.uniform_u32(n, seed)
        if kind == "dup16":
            return (inputs.uniform_u32(n, seed) & np.uint32(15)).astype(np.uint32)
        if kind == "bunched":
            u = inputs.uniform_u32(n, seed)
            return np.where((u >> 28) == 0, u, u & np.uint32(0xFFF)).astype(np.uint32)
        raise ValueError(kind)
    if kind == "uniform":
        return inputs.uniform_u64(n, seed)
    if kind == "sorted":
        return inputs.sorted_u64(n, seed)
    if kind == "reverse":
        return inputs.reverse_sorted_u64(n, seed)
    if kind == "dup16":
        return inputs.heavy_duplicates_u64(n, seed, 16)
    if kind == "equal":
        return np.full(n, np.uint64(0x1234), dtype=np.uint64)
    if kind == "zeros":
        return np.zeros(n, dtype=np.uint64)
    if kind == "max":
        return np.full(n, np.uint64(2**64 - 1), dtype=np.uint64)
    if kind == "bunched":
        # 15 of 16 keys in [0, 4096), the rest anywhere: a small subarray that
        # holds both has one bucket of most of its keys, so the bucket sort
        # turns it down and the merge sort takes it
        u = inputs.uniform_u64(n, seed)
        return np.where((u >> 60) == 0, u, u & np.uint64(0xFFF)).astype(np.uint64)
    if kind == "two":
        return np.where(inputs.uniform_u64(n, seed) & np.uint64(1), np.uint64(0),
                        np.uint64(2**64 - 1)).astype(np.uint64)
    raise ValueError(kind)


def run_and_compare(ctx, host, seed=5):
    ref = host.copy()
    oracle.quicksort(ref, seed)
    assert np.array_equal(ref, np.sort(host))  # the oracle sorts
    d = to_dev(host)
    lp.lp_quicksort(ctx, d, seed=seed)
    torch.cuda.synchronize()
    out = to_host(d, host.dtype)
    assert np.array_equal(out, ref)


# around the shared-memory sort (4096 keys), one CTA's on-chip partition
# (about 12K uint64 keys), the finishing kernel's cut (65536 keys: larger
# subarrays go through the level-synchronous levels first), several levels
SIZES = [0, 1, 2, 3, 17, 4095, 4096, 4097, 8191, 12289, 40000, 65535, 65536, 65537,
         65536 + 7, 131073, 1 << 20, (1 << 21) + 333]


@pytest.mark.parametrize("n", SIZES)
def test_uniform_u64_sizes(ctx, n):
    run_and_compare(ctx, make("uniform", n, 100 + n))


@pytest.mark.parametrize("kind", ["sorted", "reverse", "dup16", "equal", "zeros", "max", "two",
                                  "bunched"])
@pytest.mark.parametrize("n", [5000, 50001, 300000])
def test_patterns_u64(ctx, kind, n):
    run_and_compare(ctx, make(kind, n, 7 + n))


@pytest.mark.parametrize("kind", ["uniform", "dup16", "bunched"])
@pytest.mark.parametrize("n", [1, 4096, 4097, 30001, 65536, 65537, 100003, 1 << 20, 1 << 25])
def test_u32(ctx, kind, n):
    # 2^25 keys: the first levels leave open ranges that several CTAs finish
    # on chip at once (the batched engine's multi-CTA finish for 4-byte keys)
    run_and_compare(ctx, make(kind, n, 31 + n, np.uint32))


@pytest.mark.parametrize("off", [1, 3])
def test_unaligned_view(ctx, off):
    n = 200001
    host = make("uniform", n + off + 2, 9)
    d = to_dev(host)
    view = d[off:off + n]
    lp.lp_quicksort(ctx, view, seed=3)
    torch.cuda.synchronize()
    out = to_host(d, np.uint64)
    ref = host.copy()
    oracle.quicksort(ref[off:off + n], 3)
    assert np.array_equal(out, ref)  # keys outside the view unchanged


def test_seed_independent_result(ctx):
    host = make("dup16", 1 << 19, 4)
    outs = []
    for seed in (0, 1, 12345):
        d = to_dev(host)
        lp.lp_quicksort(ctx, d, seed=seed)
        outs.append(to_host(d, np.uint64))
    assert all(np.array_equal(outs[0], o) for o in outs)
    assert np.array_equal(outs[0], np.sort(host))


def test_aux_memory_small(ctx):  # the fixture builds the library; the check uses its own context
    """A context of its own (a shared one keeps the scratch of earlier, larger
    calls): lists and per-segment records of the quicksort stay well under 1%
    of the 128 MiB array, the context's fixed scratch included."""
    n = 1 << 24
    c = lp.Ctx(0)
    try:
        d = torch.empty(n, dtype=torch.int64, device="cuda")
        lp.lp_fill_uniform_u64(d, 77)
        lp.lp_quicksort(c, d, seed=1)
        key = unsigned_key(d)
        assert bool((key[1:] >= key[:-1]).all())
        assert c.aux_bytes < 0.01 * n * 8
    finally:
        c.close()


@pytest.mark.parametrize("kind", ["uniform", "sorted", "reverse", "dup16"])
def test_full_size_2pow28(ctx, kind):
    """The n = 2^28 uint64 workload: sorted, and equal to a library sort."""
    n = 1 << 28
    d = torch.empty(n, dtype=torch.int64, device="cuda")
    # the same patterns as the smaller cases, built on the device
    lp.lp_fill_uniform_u64(d, 2024)
    if kind == "sorted":
        d.copy_(unsigned_key(torch.sort(unsigned_key(d)).values))
    elif kind == "reverse":
        d.copy_(unsigned_key(torch.sort(unsigned_key(d), descending=True).values))
    elif kind == "dup16":
        d.bitwise_and_(15)
    expect = torch.sort(unsigned_key(d)).values
    lp.lp_quicksort(ctx, d, seed=11)
    got = unsigned_key(d)
    assert torch.equal(got, expect)


@pytest.mark.parametrize("kind", ["uniform", "dup16", "sorted"])
@pytest.mark.parametrize("n", [4097, 300000, (1 << 21) + 333])
def test_median_of_15_pivots(ctx, kind, n):
    """lp_quicksort_ex_* with 15 pivot samples: the same sorted output."""
    host = make(kind, n, 71 + n)
    d = to_dev(host)
    lp.lp_quicksort(ctx, d, seed=4, pivot_samples=15)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(d, host.dtype), np.sort(host))
    d32 = to_dev(make("uniform", n, n, np.uint32))
    ref32 = np.sort(to_host(d32, np.uint32))
    lp.lp_quicksort(ctx, d32, seed=4, pivot_samples=15)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(d32, np.uint32), ref32)
    with pytest.raises(lp.LPError):
        lp.lp_quicksort(ctx, d, pivot_samples=7)


@pytest.mark.parametrize("n,dtype", [((1 << 22) + 9, np.uint64), ((1 << 23) + 3, np.uint32)])
def test_tail_kernel_runs_and_sorts(ctx, n, dtype):
    """Sizes whose last levels hold few, small subarrays: the tail kernel
    sorts them (the stats say it ran) and the result equals a library sort;
    every key is sorted in shared memory at most once (keys equal to an
    equal-key item's pivot are final without a sort)."""
    host = make("uniform", n, 0x7A1 + n, dtype)
    d = to_dev(host)
    lp.lp_quicksort(ctx, d, seed=2)
    torch.cuda.synchronize()
    st = ctx.sort_stats()
    assert st["tail_items"] > 0 and st["tail_keys"] > 0, st
    assert 0.99 * n <= st["sort_keys"] <= n
    assert np.array_equal(to_host(d, dtype), np.sort(host))
