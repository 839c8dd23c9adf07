"""The allocation-free partition entry point, lp_partition_u64_noalloc.

It serves callers that cannot allocate device memory where they need a
partition (inside another allocator's callback, in latency-bound loops that
must not pay cudaMalloc's implicit synchronisation, or when a framework's pool
holds all device memory), and so cannot create an lp_ctx.  Its scratch lives in
a file-scope device array shared by all calls.  This test calls it through the
C ABI twice in a row and checks each result against the context-based entry
point on the same input and seed: the same kernels run, so the split and the
partitioned array must be identical (integers: exact).  The second call also
shows that what the first call left in the shared array does not leak into the
next result.  This file is collected last and needs no state from other tests.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_noalloc_matches_context_entry_point_twice():
    from paper_2004_12532_gb300 import binding as lp
    from paper_2004_12532_gb300 import build, inputs

    build.build()
    torch.cuda.set_device(0)
    ctx = lp.Ctx(0)
    cases = [((1 << 22) + 13, 0xA11, inputs.quantile_pivot(1, 2), lp.LP_SMOOTHED),
             ((1 << 21) + 5, 0xB22, inputs.quantile_pivot(1, 10), lp.LP_STRIDED)]
    for n, seed, pivot, variant in cases:
        host = inputs.uniform_u64(n, seed)
        a = torch.from_numpy(host.view(np.int64).copy()).cuda()
        b = a.clone()
        sa = torch.zeros(1, dtype=torch.int64, device="cuda")
        sb = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        lp.lp_partition_u64_async(ctx, a, pivot, sa, variant, seed=seed)
        lp.lp_partition_u64_noalloc(b, pivot, sb, variant, seed=seed)
        torch.cuda.synchronize()
        t = int(sb.item())
        assert t == int(sa.item())
        assert t == int((host <= np.uint64(pivot)).sum())
        assert torch.equal(a, b)
    ctx.close()
