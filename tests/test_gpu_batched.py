"""GPU parity of the batched partition engine against the serial oracle.

Segments of mixed sizes (empty, tiny, odd, one CTA's worth, several Smoothed
Striding levels), at arbitrary 8-byte offsets inside one buffer, each with its
own pivot drawn from its own keys; every segment's split and both sides'
multisets must equal the oracle's.  The graph-captured batch is replayed on
refilled keys and must give the same bytes as a fresh one-shot run.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2004_12532_gb300 import binding as lp
from paper_2004_12532_gb300 import inputs
from tests.gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2004_12532_gb300 import build
    build.build()
    c = lp.Ctx(0)
    yield c
    c.close()


def make_batch(sizes, seed):
    offs, tot = [], 1  # start at offset 1: 8-byte but not 16-byte aligned
    for n in sizes:
        offs.append(tot)
        tot += int(n) + 3
    host = inputs.uniform_u64(tot, seed)
    rng = np.random.default_rng(seed)
    pivots = []
    for o, n in zip(offs, sizes):
        pivots.append(int(host[o + rng.integers(0, n)]) if n else 0)
    return host, offs, pivots


def check_batch(out, host, offs, sizes, pivots, splits):
    for s, (o, n, p) in enumerate(zip(offs, sizes, pivots)):
        seg_in, seg_out = host[o:o + n], out[o:o + n]
        t = int(splits[s])
        ref = seg_in.copy()
        assert t == oracle.partition(ref, p), s
        pv = np.uint64(p)
        assert np.all(seg_out[:t] <= pv) and np.all(seg_out[t:] > pv), s
        assert np.array_equal(np.sort(seg_out[:t]), np.sort(ref[:t])), s
        assert np.array_equal(np.sort(seg_out[t:]), np.sort(ref[t:])), s
    # nothing outside the segments moved
    mask = np.ones(out.size, bool)
    for o, n in zip(offs, sizes):
        mask[o:o + n] = False
    assert np.array_equal(out[mask], host[mask])


SIZE_SETS = {
    "tiny": [0, 1, 2, 3, 5, 17, 100, 255, 256, 1000],
    "mixed": [0, 7, 4096, 10463, 10464, 10465, 30001, 100000, 262144 + 9, 1 << 20, 12, 2],
    "big": [(1 << 21) + 13, (1 << 22) + 1, 3 << 20],
}


@pytest.mark.parametrize("name", list(SIZE_SETS))
def test_batched_one_shot(ctx, name):
    sizes = SIZE_SETS[name]
    host, offs, pivots = make_batch(sizes, len(sizes) * 31)
    buf = to_dev(host)
    views = [buf[o:o + n] for o, n in zip(offs, sizes)]
    splits = torch.full((len(sizes),), -1, dtype=torch.int64, device="cuda")
    lp.lp_partition_batched_u64(ctx, views, pivots, splits, seed=5)
    torch.cuda.synchronize()
    check_batch(to_host(buf, np.uint64), host, offs, sizes, pivots, splits.cpu().numpy())


def test_batched_log_uniform_many(ctx):
    sizes = inputs.log_uniform_sizes(600, 0xB47C, 8, 18).tolist()
    host, offs, pivots = make_batch(sizes, 77)
    buf = to_dev(host)
    views = [buf[o:o + n] for o, n in zip(offs, sizes)]
    splits = torch.zeros(len(sizes), dtype=torch.int64, device="cuda")
    lp.lp_partition_batched_u64(ctx, views, pivots, splits, seed=9)
    torch.cuda.synchronize()
    check_batch(to_host(buf, np.uint64), host, offs, sizes, pivots, splits.cpu().numpy())


def test_batch_graph_replay_matches_one_shot(ctx):
    sizes = [3, 5000, 70000, (1 << 20) + 3, 64, 12345]
    host, offs, pivots = make_batch(sizes, 5)
    buf = to_dev(host)
    views = [buf[o:o + n] for o, n in zip(offs, sizes)]
    splits = torch.zeros(len(sizes), dtype=torch.int64, device="cuda")
    b = lp.Batch(ctx, views, pivots, splits, seed=3)
    for _ in range(2):  # replay twice on the same input
        buf.copy_(to_dev(host))
        b.launch()
        torch.cuda.synchronize()
        out = to_host(buf, np.uint64)
        check_batch(out, host, offs, sizes, pivots, splits.cpu().numpy())
    b.close()
    buf2 = to_dev(host)
    views2 = [buf2[o:o + n] for o, n in zip(offs, sizes)]
    splits2 = torch.zeros(len(sizes), dtype=torch.int64, device="cuda")
    lp.lp_partition_batched_u64(ctx, views2, pivots, splits2, seed=3)
    torch.cuda.synchronize()
    assert torch.equal(buf2, buf) and torch.equal(splits2, splits)


def test_batched_alone_equals_single(ctx):
    """A segment's result in the batch equals its result as a single call's
    multisets and split (the placement inside each side may differ)."""
    sizes = [(1 << 21) + 5, 9000, 300]
    host, offs, pivots = make_batch(sizes, 8)
    buf = to_dev(host)
    views = [buf[o:o + n] for o, n in zip(offs, sizes)]
    splits = torch.zeros(len(sizes), dtype=torch.int64, device="cuda")
    lp.lp_partition_batched_u64(ctx, views, pivots, splits, seed=1)
    torch.cuda.synchronize()
    for s, (o, n, p) in enumerate(zip(offs, sizes, pivots)):
        single = to_dev(host[o:o + n])
        t = lp.lp_partition_u64(ctx, single, p)
        assert t == int(splits[s].item())
        a = np.sort(to_host(single, np.uint64)[:t])
        bq = np.sort(to_host(buf, np.uint64)[o:o + t])
        assert np.array_equal(a, bq)


def test_autotune_and_tuned_run(ctx):
    sizes = inputs.log_uniform_sizes(64, 0x7E, 8, 20).tolist()
    best = lp.lp_autotune_batched_u64(ctx, sizes)
    assert best["line_bytes"] in (1024, 2048) and best["min_chunks"] > 0
    host, offs, pivots = make_batch(sizes, 12)
    buf = to_dev(host)
    views = [buf[o:o + n] for o, n in zip(offs, sizes)]
    splits = torch.zeros(len(sizes), dtype=torch.int64, device="cuda")
    lp.lp_partition_batched_u64(ctx, views, pivots, splits, seed=2)
    torch.cuda.synchronize()
    check_batch(to_host(buf, np.uint64), host, offs, sizes, pivots, splits.cpu().numpy())
    lp.lp_ctx_set_batch_tuning(ctx)  # back to defaults


def test_round_stats_and_streamed_keys(ctx):
    """The device-side counters: every key of every segment is streamed at
    least once, and the round record covers the launch."""
    sizes = [5, 3000, 40000, (1 << 21) + 7, 123457, 0, 64]
    host, offs, pivots = make_batch(sizes, 21)
    buf = to_dev(host)
    views = [buf[o:o + n] for o, n in zip(offs, sizes)]
    splits = torch.zeros(len(sizes), dtype=torch.int64, device="cuda")
    lp.lp_partition_batched_u64(ctx, views, pivots, splits, seed=4)
    ctx.wait()
    keys = ctx.last_batch_keys()
    rounds = ctx.last_batch_rounds()
    assert keys >= sum(n - 16 for n in sizes if n > 16)
    assert 1 <= len(rounds) <= 12 and rounds[0]["tasks"] > 0
    assert all(r["plan_ms"] >= 0 and r["task_ms"] >= 0 for r in rounds)
    check_batch(to_host(buf, np.uint64), host, offs, sizes, pivots, splits.cpu().numpy())
    b = lp.Batch(ctx, views, pivots, splits, seed=4)
    buf.copy_(to_dev(host))
    b.launch()
    b.wait()
    assert b.streamed_keys() == keys  # same segments, same seed: the same steps
    assert [r["tasks"] for r in b.round_stats()] == [r["tasks"] for r in rounds]
    b.close()


@pytest.mark.parametrize("mcr", [8, 32])
def test_residual_tuning_keeps_results_valid(ctx, mcr):
    sizes = [(1 << 22) + 5, 70000, 9000, 1 << 20]
    host, offs, pivots = make_batch(sizes, 30 + mcr)
    buf = to_dev(host)
    views = [buf[o:o + n] for o, n in zip(offs, sizes)]
    splits = torch.zeros(len(sizes), dtype=torch.int64, device="cuda")
    lp.lp_ctx_set_batch_tuning(ctx, min_chunks_residual=mcr)
    try:
        lp.lp_partition_batched_u64(ctx, views, pivots, splits, seed=2)
        torch.cuda.synchronize()
        check_batch(to_host(buf, np.uint64), host, offs, sizes, pivots, splits.cpu().numpy())
    finally:
        lp.lp_ctx_set_batch_tuning(ctx)


@pytest.mark.parametrize("onchip_slices", [0, 4])
def test_multi_cta_finish_same_in_any_batch(ctx, onchip_slices):
    """Segments large enough that their first step leaves open ranges of
    several CTAs' shared memory, which several CTAs finish on chip at once
    (each slice waits for the others of its range to be staged): each result
    equals the oracle's, and is byte for byte the result of the same segment
    at the same place in a batch of its own.  At most 4 slices per range cut
    the windows of their counts to 16 slices, so the finishes take several
    windows."""
    sizes = [(1 << 24) + 3] * 3 + [(1 << 23) + 1001] * 4 + [5000, 70001]
    host, offs, pivots = make_batch(sizes, 99)
    lp.lp_ctx_set_batch_tuning(ctx, onchip_slices=onchip_slices)
    try:
        buf = to_dev(host)
        views = [buf[o:o + n] for o, n in zip(offs, sizes)]
        splits = torch.zeros(len(sizes), dtype=torch.int64, device="cuda")
        lp.lp_partition_batched_u64(ctx, views, pivots, splits, seed=6)
        torch.cuda.synchronize()
        out = to_host(buf, np.uint64)
        check_batch(out, host, offs, sizes, pivots, splits.cpu().numpy())
        for s in (0, 4):
            o, n = offs[s], sizes[s]
            # the same offset modulo 16 bytes as in the batch buffer, so the
            # same unaligned head and body
            k = o % 2
            whole = to_dev(host[o - k:o + n])
            alone = whole[k:]
            empty = whole[0:0]
            sp = torch.zeros(s + 1, dtype=torch.int64, device="cuda")
            lp.lp_partition_batched_u64(ctx, [empty] * s + [alone], [0] * s + [pivots[s]], sp,
                                        seed=6)
            torch.cuda.synchronize()
            assert int(sp[s].item()) == int(splits[s].item())
            assert np.array_equal(to_host(alone, np.uint64), out[o:o + n])
    finally:
        lp.lp_ctx_set_batch_tuning(ctx)


def test_many_multi_cta_finishes_in_one_round(ctx):
    """Forty segments of about 2^20 keys: their first steps leave residual
    ranges of a few CTAs' shared memory each, all finished on chip in the same
    round by CTAs that take their slices from one counter; with at most 3
    slices per range (windows of 12 slices) the same batch runs through many
    windows.  Both give oracle-exact splits and sides."""
    sizes = [(1 << 20) + 17 * i for i in range(40)]
    host, offs, pivots = make_batch(sizes, 123)
    for slices in (0, 3):
        lp.lp_ctx_set_batch_tuning(ctx, onchip_slices=slices)
        try:
            buf = to_dev(host)
            views = [buf[o:o + n] for o, n in zip(offs, sizes)]
            splits = torch.zeros(len(sizes), dtype=torch.int64, device="cuda")
            lp.lp_partition_batched_u64(ctx, views, pivots, splits, seed=11)
            torch.cuda.synchronize()
            check_batch(to_host(buf, np.uint64), host, offs, sizes, pivots,
                        splits.cpu().numpy())
        finally:
            lp.lp_ctx_set_batch_tuning(ctx)
