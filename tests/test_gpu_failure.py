"""Failure detection without a GPU fault: the library's bounded waits give up
and report (a wait on an mbarrier phase nothing completes, a grid barrier for
a CTA that does not exist), the device stays usable, and a partition run
afterwards is still correct."""
import numpy as np
import pytest

import oracle
from paper_2004_12532_gb300 import binding as lp
from paper_2004_12532_gb300 import inputs
from tests.gpu_util import check_partition, to_dev, to_host

pytestmark = pytest.mark.gpu


def test_bounded_waits_give_up_and_device_stays_usable():
    from paper_2004_12532_gb300 import build
    build.build()
    assert lp.lp_selftest_bounded_waits(0) == (1, 1)
    ctx = lp.Ctx(0)
    host = inputs.uniform_u64(1 << 20, 3)
    d = to_dev(host)
    pv = inputs.quantile_pivot(1, 2)
    t = lp.lp_partition_u64(ctx, d, pv)
    check_partition(to_host(d, np.uint64), host, t, oracle.count(host, pv), pv)
    ctx.wait()
    ctx.close()
