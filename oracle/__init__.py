"""ctypes view of the C oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU legs of bench.py.  The product package never imports this module, and this
module never imports the product package.  Arrays are numpy, modified in place.
"""
import ctypes as C

import numpy as np

from . import build as _build

_u64 = C.c_uint64
_u32 = C.c_uint32
_p = C.c_void_p

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        sig = {
            "or_stream": (_u64, [_u64, _u64]),
            "or_range": (_u64, [_u64, _u64]),
            "or_count_u64": (_u64, [_p, _u64, _u64]),
            "or_count_u32": (_u64, [_p, _u64, _u32]),
            "or_partition_u64": (_u64, [_p, _u64, _u64]),
            "or_partition_u32": (_u64, [_p, _u64, _u32]),
            "or_partition_kv_u64": (_u64, [_p, _p, _u64, _u64]),
            "or_partition_rows_u64": (None, [_p, _u64, _u64, _u64, _p]),
            "or_draw_X": (None, [_u64, _u64, _u64, _u64, _p]),
            "or_num_chunks": (_u64, [_u64, _u64, _u64]),
            "or_smoothed_step_u64": (C.c_int, [_p, _u64, _u64, _u64, _u64, _p, _p, _p, _p, _p]),
            "or_smoothed_step_u32": (C.c_int, [_p, _u64, _u32, _u64, _u64, _p, _p, _p, _p, _p]),
            "or_smoothed_partition_u64": (_u64, [_p, _u64, _u64, _u64, _u64, _u64, _u64, _u64, _p]),
            "or_strided_partition_u64": (_u64, [_p, _u64, _u64, _u64, _u64]),
            "or_make_successor_heavy_u64": (None, [_p, _u64, _u64, C.c_int]),
            "or_block_prefix_u64": (_u64, [_p, _u64, _u64, C.c_int, _u64, _p]),
            "or_reorder_u64": (None, [_p, _u64, _u64, C.c_int, _u64, _p]),
            "or_lowspace_partition_u64": (_u64, [_p, _u64, _u64, _u64]),
            "or_bits_for": (_u64, [_u64]),
            "or_bitstore_encode_u64": (None, [_p, _u64, _u64, C.c_int]),
            "or_bitstore_decode_u64": (_u64, [_p, _u64, C.c_int]),
            "or_implicit_prefix_u64": (_u64, [_p, _u64, _u64, _u64, _p]),
            "or_implicit_partition_u64": (_u64, [_p, _u64, _u64, _u64]),
            "or_quicksort_u64": (None, [_p, _u64, _u64]),
            "or_quicksort_u32": (None, [_p, _u64, _u64]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _check(a, dt):
    if a.dtype != dt or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("expected a contiguous %s array" % dt)


def stream(seed, k):
    return int(lib().or_stream(seed & (2**64 - 1), k & (2**64 - 1)))


def rng_range(r, g):
    return int(lib().or_range(r, g))


def count(a, pivot):
    if a.dtype == np.uint64:
        return int(lib().or_count_u64(_ptr(a), a.size, int(pivot)))
    _check(a, np.uint32)
    return int(lib().or_count_u32(_ptr(a), a.size, int(pivot)))


def partition(a, pivot):
    """Serial in-place partition by [x <= pivot]; returns the split t."""
    if a.dtype == np.uint64:
        return int(lib().or_partition_u64(_ptr(a), a.size, int(pivot)))
    _check(a, np.uint32)
    return int(lib().or_partition_u32(_ptr(a), a.size, int(pivot)))


def partition_kv(k, v, pivot):
    _check(k, np.uint64)
    _check(v, np.uint64)
    assert k.size == v.size
    return int(lib().or_partition_kv_u64(_ptr(k), _ptr(v), k.size, int(pivot)))


def partition_rows(a2d, pivot):
    _check(a2d, np.uint64)
    rows, ln = a2d.shape
    t = np.zeros(rows, dtype=np.uint64)
    lib().or_partition_rows_u64(_ptr(a2d), rows, ln, int(pivot), _ptr(t))
    return t


def draw_X(seed, level, s, g):
    X = np.zeros(max(s, 1), dtype=np.uint64)
    lib().or_draw_X(seed, level, s, g, _ptr(X))
    return X[:s]


def num_chunks(n, b, g):
    return int(lib().or_num_chunks(n, b, g))


def smoothed_step(a, pivot, b, g, X):
    """One Partial Partition Step on the whole of a; returns (k, v, vmin, vmax)."""
    X = np.ascontiguousarray(X, dtype=np.uint64)
    s = num_chunks(a.size, b, g)
    assert X.size >= s
    Xp = X if X.size else np.zeros(1, dtype=np.uint64)
    k = np.zeros(g, dtype=np.uint64)
    v = np.zeros(g, dtype=np.uint64)
    vmin = C.c_uint64()
    vmax = C.c_uint64()
    f = lib().or_smoothed_step_u64 if a.dtype == np.uint64 else lib().or_smoothed_step_u32
    if a.dtype != np.uint64:
        _check(a, np.uint32)
    rc = f(_ptr(a), a.size, int(pivot), b, g, _ptr(Xp), _ptr(k), _ptr(v),
           C.byref(vmin), C.byref(vmax))
    if rc != 0:
        raise ValueError("bad smoothed step arguments")
    return k, v, int(vmin.value), int(vmax.value)


def smoothed_partition(a, pivot, seed, b=64, gmax=64, smin=16, base=256):
    _check(a, np.uint64)
    lv = C.c_uint64()
    t = lib().or_smoothed_partition_u64(_ptr(a), a.size, int(pivot), seed, b, gmax,
                                        smin, base, C.byref(lv))
    return int(t), int(lv.value)


def strided_partition(a, pivot, b, g):
    _check(a, np.uint64)
    return int(lib().or_strided_partition_u64(_ptr(a), a.size, int(pivot), b, g))


def make_successor_heavy(a, pivot, flip=0):
    _check(a, np.uint64)
    lib().or_make_successor_heavy_u64(_ptr(a), a.size, int(pivot), int(flip))


def block_prefix(a, pivot, B, flip=0):
    _check(a, np.uint64)
    v = np.zeros(max(a.size // B, 1), dtype=np.uint64)
    nb = lib().or_block_prefix_u64(_ptr(a), a.size, int(pivot), int(flip), B, _ptr(v))
    return v[:nb]


def reorder(a, pivot, B, v, flip=0):
    _check(a, np.uint64)
    v = np.ascontiguousarray(v, dtype=np.uint64)
    vp = v if v.size else np.zeros(1, dtype=np.uint64)
    lib().or_reorder_u64(_ptr(a), a.size, int(pivot), int(flip), B, _ptr(vp))


def lowspace_partition(a, pivot, B=4096):
    _check(a, np.uint64)
    return int(lib().or_lowspace_partition_u64(_ptr(a), a.size, int(pivot), B))


def bits_for(n):
    return int(lib().or_bits_for(n))


def bitstore_encode(x, L, v, first):
    """Encode v in x[:4L+2] (modified in place)."""
    _check(x, np.uint64)
    assert x.size >= 4 * L + 2
    lib().or_bitstore_encode_u64(_ptr(x), L, int(v), 1 if first else 0)


def bitstore_decode(x, L, restore=True):
    _check(x, np.uint64)
    assert x.size >= 4 * L + 2
    return int(lib().or_bitstore_decode_u64(_ptr(x), L, 1 if restore else 0))


def implicit_prefix(a, pivot, B):
    """Returns (t, flip); a is left with every block's value encoded."""
    _check(a, np.uint64)
    f = C.c_int(0)
    t = int(lib().or_implicit_prefix_u64(_ptr(a), a.size, int(pivot), B, C.byref(f)))
    return t, int(f.value)


def implicit_partition(a, pivot, B):
    _check(a, np.uint64)
    return int(lib().or_implicit_partition_u64(_ptr(a), a.size, int(pivot), B))


def quicksort(a, seed=0):
    if a.dtype == np.uint64:
        lib().or_quicksort_u64(_ptr(a), a.size, seed)
    else:
        _check(a, np.uint32)
        lib().or_quicksort_u32(_ptr(a), a.size, seed)
