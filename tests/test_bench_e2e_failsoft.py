"""bench.py's end-to-end leg fails soft, no GPU: when the pinned host buffers
cannot be had (here: no accelerator at all), the leg reports itself
unavailable instead of raising, after joining the rank reduction."""
import types

import bench
from paper_2004_12532_gb300 import binding


def test_e2e_leg_unavailable_without_pinned_memory():
    args = types.SimpleNamespace(e2e_steps=2)
    out = bench.e2e_leg(args, binding, None, None, None, 5, None, 1 << 10, 0, None)
    assert out["value"] is None and out["unavailable"]
