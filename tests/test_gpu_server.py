"""GPU tests of the serving engine (continuous batching of partition and sort
requests under a slot limit and a device-memory budget).

Every finished request is checked against the oracle: a partition's split
and both sides' multisets, a sort's bytes.  A request's result must be the
same, byte for byte, when it runs alone and when it runs in a mix; the budget
must never be exceeded; the open-loop driver must finish every request with
done >= admit >= arrival; the one-at-a-time baseline must give the same
splits.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2004_12532_gb300 import binding as lp
from paper_2004_12532_gb300 import inputs
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu

P, S = lp.LP_REQ_PARTITION, lp.LP_REQ_SORT


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2004_12532_gb300 import build
    build.build()


def host_keys(n, bits, seed):
    return inputs.uniform_u64(n, seed) if bits == 64 else inputs.uniform_u32(n, seed)


def mixed_requests(seed, count=40):
    rng = np.random.default_rng(seed)
    sizes = [0, 1, 2, 3, 100, 4096, 4097, 5000, 70001, 300000, 1 << 20]
    reqs = []
    for i in range(count):
        kind = S if rng.random() < 0.4 else P
        bits = 64 if rng.random() < 0.5 else 32
        n = int(sizes[i % len(sizes)] if i < len(sizes) else rng.integers(0, 400000))
        keys = host_keys(n, bits, 1000 + i)
        if bits == 32 and kind == S and i % 3 == 0:
            keys = keys & np.uint32(15)  # heavy duplicates
        if bits == 64 and kind == S and i % 3 == 1:
            # 15 of 16 keys in [0, 4096): small subarrays the merge sort takes
            keys = np.where((keys >> 60) == 0, keys, keys & np.uint64(0xFFF)).astype(np.uint64)
        pivot = int(keys[rng.integers(0, n)]) if n else 0
        reqs.append((kind, bits, n, pivot, 5000 + i, keys))
    return reqs


def check_result(kind, bits, n, pivot, keys, out, split):
    if kind == S:
        assert np.array_equal(out, np.sort(keys))
        return
    ref = keys.copy()
    t = oracle.partition(ref, pivot)
    assert split == t
    p = out.dtype.type(pivot)
    assert np.all(out[:t] <= p) and np.all(out[t:] > p)
    assert np.array_equal(np.sort(out[:t]), np.sort(ref[:t]))
    assert np.array_equal(np.sort(out[t:]), np.sort(ref[t:]))


def drain(srv, expect):
    done = []
    for _ in range(100000):
        srv.step()
        done += srv.poll()
        if len(done) >= expect:
            return done
    raise AssertionError("requests did not finish")


def test_mixed_requests_match_oracle():
    reqs = mixed_requests(1)
    srv = lp.Server(budget_bytes=1 << 30, max_slots=16, keep_results=True)
    srcs, ids = {}, {}
    for k, (kind, bits, n, pivot, seed, keys) in enumerate(reqs):
        src = to_dev(keys) if n else None  # kept allocated until admission
        torch.cuda.synchronize()
        i = srv.submit(kind, bits, n, pivot=pivot, seed=seed, src=src)
        srcs[i] = src
        ids[i] = k
    done = drain(srv, len(reqs))
    torch.cuda.synchronize()
    assert sorted(c["id"] for c in done) == sorted(ids)
    for c in done:
        kind, bits, n, pivot, seed, keys = reqs[ids[c["id"]]]
        assert c["arrival_s"] <= c["admit_s"] <= c["done_s"]
        out = srv.fetch(c["id"], n, bits)
        check_result(kind, bits, n, pivot, keys, out, c["split"])
        srv.release(c["id"])
    st = srv.stats()
    assert st["in_use_bytes"] == 0 and st["completed"] == len(reqs)
    assert st["peak_bytes"] <= st["budget_bytes"]
    srv.close()


def test_result_same_alone_and_in_mix():
    reqs = mixed_requests(2, count=24)
    mix = lp.Server(budget_bytes=1 << 30, max_slots=32, keep_results=True, seed=9)
    ids = []
    # a request's source keys must stay allocated until it is admitted
    srcs = [to_dev(r[5]) if r[2] else None for r in reqs]
    torch.cuda.synchronize()
    for (kind, bits, n, pivot, seed, keys), src in zip(reqs, srcs):
        ids.append(mix.submit(kind, bits, n, pivot=pivot, seed=seed, src=src))
    drain(mix, len(reqs))
    in_mix = [mix.fetch(i, r[2], r[1]) for i, r in zip(ids, reqs)]
    mix.close()
    for k, (kind, bits, n, pivot, seed, keys) in enumerate(reqs):
        alone = lp.Server(budget_bytes=1 << 28, max_slots=4, keep_results=True, seed=9)
        i = alone.submit(kind, bits, n, pivot=pivot, seed=seed, src=srcs[k])
        c = drain(alone, 1)[0]
        out = alone.fetch(i, n, bits)
        assert np.array_equal(out, in_mix[k]), (k, kind, bits, n)
        check_result(kind, bits, n, pivot, keys, out, c["split"])
        alone.close()


def test_budget_limits_admission():
    # each request holds 8 MiB of keys; a 20 MiB budget admits two at a time
    srv = lp.Server(budget_bytes=20 << 20, max_slots=8, keep_results=False)
    n = 1 << 20
    for i in range(6):
        srv.submit(P, 64, n, pivot=(1 << 63) - 1, seed=i)
    done = []
    for _ in range(1000):
        srv.step()
        st = srv.stats()
        assert st["in_use_bytes"] <= st["budget_bytes"]
        done += srv.poll()
        if len(done) == 6:
            break
    assert len(done) == 6
    assert srv.stats()["peak_bytes"] <= 20 << 20
    # FIFO: admission times are in submission order
    adm = [c["admit_s"] for c in sorted(done, key=lambda c: c["id"])]
    assert adm == sorted(adm)
    srv.close()


def test_invalid_requests_rejected():
    srv = lp.Server(budget_bytes=1 << 20, max_slots=4)
    with pytest.raises(lp.LPError):
        srv.submit(P, 16, 10)
    with pytest.raises(lp.LPError):
        srv.submit(7, 64, 10)
    with pytest.raises(lp.LPError):
        srv.submit(P, 64, 1 << 20)  # 8 MiB > 1 MiB budget
    srv.close()


def poisson_requests(count, rate, seed, lo_log2=10, hi_log2=20):
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    sizes = inputs.log_uniform_sizes(count, seed, lo_log2, hi_log2)
    reqs = []
    for i in range(count):
        kind = S if rng.random() < 0.3 else P
        bits = 64 if rng.random() < 0.5 else 32
        pivot = inputs.quantile_pivot(int(rng.integers(1, 100)), 100, bits)
        reqs.append(lp.Server.request(kind, bits, int(sizes[i]), pivot, 77 + i, None,
                                      float(t[i])))
    return reqs


def test_open_loop_run_and_one_at_a_time():
    reqs = poisson_requests(300, 3000.0, 5)
    srv = lp.Server(budget_bytes=2 << 30, max_slots=64)
    out = srv.run(reqs)
    for r, c in zip(reqs, out):
        assert c["n"] == r.n and c["kind"] == r.kind
        assert c["arrival_s"] <= c["admit_s"] + 1e-9 and c["admit_s"] <= c["done_s"]
    # the same partitions give the same splits one at a time (plain calls)
    base = srv.run(reqs, mode=lp.LP_SERVE_ONE_AT_A_TIME)
    for r, a, b in zip(reqs, out, base):
        if r.kind == P:
            assert a["split"] == b["split"]
    # splits agree with the oracle on the generated keys
    for r, c in list(zip(reqs, out))[:40]:
        if r.kind == P:
            if r.key_bits == 64:
                d = torch.empty(r.n, dtype=torch.int64, device="cuda")
                lp.lp_fill_uniform_u64(d, r.seed)
                keys = d.cpu().numpy().view(np.uint64)
            else:
                d = torch.empty(r.n, dtype=torch.int32, device="cuda")
                lp.lp_fill_uniform_u32(d, r.seed)
                keys = d.cpu().numpy().view(np.uint32)
            assert c["split"] == oracle.count(keys, r.pivot)
    st = srv.stats()
    assert st["completed"] == 2 * len(reqs)
    assert sum(srv.streamed_keys()) > 0
    srv.close()


def device_keys(n, bits, seed):
    """A request's keys as the server generates them from its seed (src=None):
    lp_fill_uniform_*, copied to the host."""
    d = torch.empty(n, dtype=torch.int64 if bits == 64 else torch.int32, device="cuda")
    (lp.lp_fill_uniform_u64 if bits == 64 else lp.lp_fill_uniform_u32)(d, seed)
    return d.cpu().numpy().view(np.uint64 if bits == 64 else np.uint32)


def test_large_requests_same_alone_and_in_mix():
    """The serving workload's large requests (2^24 .. 2^26 keys, both widths):
    multi-level Smoothed Striding steps and multi-CTA finishes for partitions,
    deep quicksort levels for sorts, all inside one mix with small requests.
    Each result equals, byte for byte, the same request run alone, and the
    oracle's result (a partition's split and sides; a sort's bytes)."""
    big = [(P, 64, 1 << 26), (S, 64, 1 << 24), (P, 32, (1 << 25) + 3), (S, 32, 1 << 26),
           (P, 64, (1 << 24) + 1), (S, 64, (1 << 25) + 5)]
    small = [(P, 32, 5000), (S, 64, 70001), (P, 64, 300000), (S, 32, 4097)]
    reqs = []
    for i, (kind, bits, n) in enumerate(big + small):
        q = (1, 100) if i % 3 == 0 else ((1, 2) if i % 3 == 1 else (99, 100))
        reqs.append((kind, bits, n, inputs.quantile_pivot(q[0], q[1], bits), 0xB16 + i))
    mix = lp.Server(budget_bytes=4 << 30, max_slots=16, keep_results=True, seed=11)
    ids = [mix.submit(kind, bits, n, pivot=pivot, seed=seed)
           for kind, bits, n, pivot, seed in reqs]
    drain(mix, len(reqs))
    in_mix = [mix.fetch(i, r[2], r[1]) for i, r in zip(ids, reqs)]
    assert mix.stats()["peak_bytes"] <= 4 << 30
    mix.close()
    for k, (kind, bits, n, pivot, seed) in enumerate(reqs):
        alone = lp.Server(budget_bytes=1 << 30, max_slots=2, keep_results=True, seed=11)
        i = alone.submit(kind, bits, n, pivot=pivot, seed=seed)
        c = drain(alone, 1)[0]
        out = alone.fetch(i, n, bits)
        alone.close()
        assert np.array_equal(out, in_mix[k]), (k, kind, bits, n)
        check_result(kind, bits, n, pivot, device_keys(n, bits, seed), out, c["split"])
