"""The allocation-free partition entry point, lp_partition_u64_noalloc.

It serves callers that cannot allocate device memory where they need a
partition (inside another allocator's callback, in latency-bound loops that
must not pay cudaMalloc's implicit synchronisation, or when a framework's pool
holds all device memory), and so cannot create an lp_ctx.  Its scratch lives in
a file-scope device array shared by all calls.

Each case calls it through the C ABI twice in a row (the second call shows that
what the first left in the shared array does not leak into the next result)
and checks it against the oracle: the split equals the oracle's and each side
holds the oracle's side as a multiset (integers: exact).  For LP_SMOOTHED on
arrays that need no handoff, both entry points run the same kernels, so the
partitioned array must also equal the context-based entry point's byte for
byte.  LP_STRIDED differs by design above on-chip size (the context path
cleans the Strided step's open range with the low-space partition, this one
with the Smoothed Striding recursion), so there only the oracle comparison
applies; 2^23 + 5 keys are more than all CTAs' shared memory holds, so the
recursion really runs.  This file is collected last and needs no state from
other tests.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _sides_match_oracle(orc, out, host, t, pivot):
    ref = host.copy()
    t_ref = orc.partition(ref, pivot)
    assert t == t_ref, (t, t_ref)
    assert np.array_equal(np.sort(out[:t]), np.sort(ref[:t_ref]))
    assert np.array_equal(np.sort(out[t:]), np.sort(ref[t_ref:]))


@pytest.mark.parametrize("n,seed,q,variant,same_kernels", [
    ((1 << 22) + 13, 0xA11, (1, 2), "smoothed", True),
    ((1 << 21) + 5, 0xB22, (1, 10), "strided", True),
    ((1 << 23) + 5, 0xC33, (1, 100), "strided", False),
    ((1 << 23) + 5, 0xD44, (1, 2), "strided", False),
])
def test_noalloc_twice_against_oracle(orc, n, seed, q, variant, same_kernels):
    from paper_2004_12532_gb300 import binding as lp
    from paper_2004_12532_gb300 import build, inputs

    build.build()
    torch.cuda.set_device(0)
    v = {"smoothed": lp.LP_SMOOTHED, "strided": lp.LP_STRIDED}[variant]
    pivot = inputs.quantile_pivot(q[0], q[1])
    ctx = lp.Ctx(0)
    for call in range(2):
        host = inputs.uniform_u64(n, seed + call)
        b = torch.from_numpy(host.view(np.int64).copy()).cuda()
        sb = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        lp.lp_partition_u64_noalloc(b, pivot, sb, v, seed=seed + call)
        torch.cuda.synchronize()
        t = int(sb.item())
        out = b.cpu().numpy().view(np.uint64)
        _sides_match_oracle(orc, out, host, t, pivot)
        if same_kernels:
            a = torch.from_numpy(host.view(np.int64).copy()).cuda()
            sa = torch.zeros(1, dtype=torch.int64, device="cuda")
            lp.lp_partition_u64_async(ctx, a, pivot, sa, v, seed=seed + call)
            torch.cuda.synchronize()
            assert int(sa.item()) == t
            assert torch.equal(a, b)
    ctx.close()
