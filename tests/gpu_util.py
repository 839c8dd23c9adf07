"""Shared helpers of the GPU parity tests (no oracle arithmetic here)."""
import numpy as np
import torch

SIGN = np.uint64(1 << 63)


def to_dev(a: np.ndarray) -> torch.Tensor:
    """Copy a uint64 / uint32 numpy array to the GPU as same-width signed ints."""
    if a.dtype == np.uint64:
        return torch.from_numpy(a.view(np.int64).copy()).cuda()
    assert a.dtype == np.uint32
    return torch.from_numpy(a.view(np.int32).copy()).cuda()


def to_host(t: torch.Tensor, dtype) -> np.ndarray:
    return t.cpu().numpy().view(dtype)


def check_partition(out: np.ndarray, inp: np.ndarray, t: int, t_ref: int, pivot: int):
    """Split equal to the oracle's; both sides equal as multisets to the
    oracle's (equivalently: postcondition holds and out permutes inp)."""
    assert t == t_ref, (t, t_ref)
    p = out.dtype.type(pivot)
    assert np.all(out[:t] <= p), "a successor left of the split"
    assert np.all(out[t:] > p), "a predecessor right of the split"
    assert np.array_equal(np.sort(out[:t]), np.sort(inp[inp <= p]))
    assert np.array_equal(np.sort(out[t:]), np.sort(inp[inp > p]))


def unsigned_key(t: torch.Tensor) -> torch.Tensor:
    """Signed view whose order matches unsigned order of the same bits."""
    if t.dtype == torch.int64:
        return t ^ torch.tensor(-(1 << 63), dtype=torch.int64, device=t.device)
    return t ^ torch.tensor(-(1 << 31), dtype=torch.int32, device=t.device)
