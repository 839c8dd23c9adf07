"""Host logic of bench.py's in-run parity checks, no GPU: the multiset
fingerprint is the same for any permutation of the keys (or of the (key,
payload) pairs) and changes when one key changes; the predicate count uses the
unsigned order of the bits for both widths; the postcondition check catches a
key on the wrong side.  CPU torch tensors stand in for device ones."""
import numpy as np
import torch

import bench


def _t64(a):
    return torch.from_numpy(a.view(np.int64).copy())


def _t32(a):
    return torch.from_numpy(a.view(np.int32).copy())


def test_fingerprint_permutation_invariant():
    rng = np.random.default_rng(5)
    a = rng.integers(0, 2**64, size=10007, dtype=np.uint64)
    p = rng.permutation(a.size)
    assert bench.fingerprint(_t64(a)) == bench.fingerprint(_t64(a[p]))
    b = a.copy()
    b[123] ^= np.uint64(1 << 40)
    assert bench.fingerprint(_t64(a)) != bench.fingerprint(_t64(b))
    # pairs: the same keys with the payloads permuted differently differ
    v = np.arange(a.size, dtype=np.uint64)
    assert bench.fingerprint(_t64(a), _t64(v)) == bench.fingerprint(_t64(a[p]), _t64(v[p]))
    q = p.copy()
    q[[0, 1]] = q[[1, 0]]
    assert bench.fingerprint(_t64(a), _t64(v)) != bench.fingerprint(_t64(a[p]), _t64(v[q]))
    c = rng.integers(0, 2**32, size=999, dtype=np.uint32)
    assert bench.fingerprint(_t32(c)) == bench.fingerprint(_t32(c[::-1].copy()))


def test_count_le_unsigned_order():
    a = np.array([0, 1, 2**63 - 1, 2**63, 2**64 - 1, 5], dtype=np.uint64)
    for pivot in [0, 1, 2**63 - 1, 2**63, 2**64 - 1]:
        assert bench.count_le(_t64(a), pivot) == int((a <= np.uint64(pivot)).sum())
    c = np.array([0, 2**31 - 1, 2**31, 2**32 - 1, 7], dtype=np.uint32)
    for pivot in [0, 2**31 - 1, 2**31, 2**32 - 1]:
        assert bench.count_le(_t32(c), pivot) == int((c <= np.uint32(pivot)).sum())


def test_partition_holds():
    a = np.array([3, 1, 2, 9, 8, 2**63 + 5], dtype=np.uint64)
    assert bench.partition_holds(_t64(a), 3, 3)
    b = a.copy()
    b[[2, 3]] = b[[3, 2]]
    assert not bench.partition_holds(_t64(b), 3, 3)
    assert bench.partition_holds(_t64(a), 0, 0)  # no key <= 0: t = 0 is the split
    z = np.array([4, 0, 7], dtype=np.uint64)
    assert not bench.partition_holds(_t64(z), 0, 0)  # a 0 right of the split
    assert bench.partition_holds(_t64(np.sort(a)), 6, 2**64 - 1)
