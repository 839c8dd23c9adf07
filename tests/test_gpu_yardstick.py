"""GPU tests of the out-of-place yardsticks timed beside the in-place
partition (libyardstick.so; never called by libpartition): the paper's
Standard linear-space partition (Sec. 2) and CUB's DevicePartition::If.

Both are stable partitions, so besides the oracle's split and side multisets
each side must equal the input's predecessors (successors) in input order --
for CUB the successors come out reversed, as its documentation states.
"""
import ctypes as C
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2004_12532_gb300 import inputs
from tests.gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def yard():
    from paper_2004_12532_gb300 import build
    build.build()
    path = os.path.join(os.path.dirname(build.LIB), "libyardstick.so")
    L = C.CDLL(path)
    L.yd_standard_scratch_words.restype = C.c_uint64
    L.yd_standard_scratch_words.argtypes = [C.c_uint64]
    L.yd_standard_partition_u64.restype = C.c_int
    L.yd_standard_partition_u64.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, C.c_void_p,
                                            C.c_void_p, C.c_void_p]
    L.yd_cub_partition_temp_bytes.restype = C.c_int
    L.yd_cub_partition_temp_bytes.argtypes = [C.c_uint64, C.POINTER(C.c_size_t)]
    L.yd_cub_partition_u64.restype = C.c_int
    L.yd_cub_partition_u64.argtypes = [C.c_void_p, C.c_void_p, C.c_uint64, C.c_uint64,
                                       C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]
    return L


def stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


CASES = [(0, (1, 2)), (1, (1, 2)), (4095, (1, 3)), (4096, (1, 2)), (4097, (99, 100)),
         ((1 << 20) + 3, (1, 100)), ((1 << 24) + 5, (1, 2)), ((1 << 22) + 1, (0, 1)),
         ((1 << 22) + 7, (1, 1))]


@pytest.mark.parametrize("n,q", CASES)
def test_standard_partition(yard, n, q):
    host = inputs.uniform_u64(n, 0x57D + n)
    pivot = inputs.quantile_pivot(q[0], q[1])
    dev = to_dev(host) if n else torch.empty(0, dtype=torch.int64, device="cuda")
    scratch = torch.empty(max(1, yard.yd_standard_scratch_words(n)), dtype=torch.int64,
                          device="cuda")
    d = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    assert yard.yd_standard_partition_u64(dev.data_ptr(), n, pivot, scratch.data_ptr(),
                                          d.data_ptr(), stream()) == 0
    torch.cuda.synchronize()
    t = int(d.item())
    ref = host.copy()
    assert t == oracle.partition(ref, pivot)
    out = to_host(dev, np.uint64)
    assert np.array_equal(np.sort(out[:t]), np.sort(ref[:t]))
    assert np.array_equal(np.sort(out[t:]), np.sort(ref[t:]))
    p = np.uint64(pivot)
    assert np.array_equal(out[:t], host[host <= p]) and np.array_equal(out[t:], host[host > p])


@pytest.mark.parametrize("n,q", CASES[1:7])
def test_cub_partition(yard, n, q):
    host = inputs.uniform_u64(n, 0xCB + n)
    pivot = inputs.quantile_pivot(q[0], q[1])
    dev = to_dev(host)
    out = torch.empty_like(dev)
    tb = C.c_size_t()
    assert yard.yd_cub_partition_temp_bytes(n, C.byref(tb)) == 0
    tmp = torch.empty(max(1, tb.value), dtype=torch.uint8, device="cuda")
    sel = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert yard.yd_cub_partition_u64(dev.data_ptr(), out.data_ptr(), n, pivot, sel.data_ptr(),
                                     tmp.data_ptr(), tb.value, stream()) == 0
    torch.cuda.synchronize()
    t = int(sel.item())
    ref = host.copy()
    assert t == oracle.partition(ref, pivot)
    o = to_host(out, np.uint64)
    p = np.uint64(pivot)
    assert np.array_equal(o[:t], host[host <= p])
    assert np.array_equal(o[t:], host[host > p][::-1])
