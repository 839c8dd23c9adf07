"""Thin ctypes binding of libpartition's C ABI (include/libpartition.h).

Argument marshalling only: every function here forwards to the function of
the same name in libpartition.so, passing a torch CUDA tensor's device pointer,
its element count and the current CUDA stream.  No computation happens here,
and there is no CPU fallback: if the library is missing, the first call raises.
"""
import ctypes as C
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpartition.so")

LP_OK = 0
LP_ERR_INVALID_ARG = 1
LP_ERR_MISALIGNED = 2
LP_ERR_OOM = 3
LP_ERR_BUDGET = 4
LP_ERR_TIMEOUT = 5
LP_ERR_CUDA = 6
LP_ERR_INTERNAL = 7

LP_SMOOTHED = 0
LP_STRIDED = 1
LP_LOWSPACE = 2
LP_HYBRID = 3
LP_MAX_LEVELS = 10

_u64 = C.c_uint64
_u32 = C.c_uint32
_p = C.c_void_p
_i = C.c_int
_pu64 = C.POINTER(C.c_uint64)

class lp_segment_u64(C.Structure):
    _fields_ = [("keys", C.c_void_p), ("n", C.c_uint64), ("pivot", C.c_uint64)]


class lp_batch_tuning(C.Structure):
    _fields_ = [("ctas", C.c_uint32), ("line_bytes", C.c_uint32), ("min_chunks", C.c_uint32),
                ("group_workers", C.c_uint32), ("min_chunks_residual", C.c_uint32),
                ("onchip_slices", C.c_uint32)]


class lp_sort_stats(C.Structure):
    _fields_ = [("levels", C.c_uint32), ("timed", C.c_uint32), ("partition_keys", C.c_uint64),
                ("sort_keys", C.c_uint64), ("partition_ms", C.c_float), ("sort_ms", C.c_float),
                ("tail_items", C.c_uint32), ("tail_ms", C.c_float), ("tail_keys", C.c_uint64)]


class lp_server_config(C.Structure):
    _fields_ = [("budget_bytes", C.c_uint64), ("max_slots", C.c_uint32),
                ("max_segments", C.c_uint32), ("seed", C.c_uint64),
                ("keep_results", C.c_uint32), ("timing", C.c_uint32)]


class lp_request(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("key_bits", C.c_uint32), ("n", C.c_uint64),
                ("pivot", C.c_uint64), ("seed", C.c_uint64), ("d_src", C.c_void_p),
                ("arrival_s", C.c_double)]


class lp_completion(C.Structure):
    _fields_ = [("id", C.c_uint64), ("kind", C.c_uint32), ("key_bits", C.c_uint32),
                ("n", C.c_uint64), ("split", C.c_uint64), ("arrival_s", C.c_double),
                ("admit_s", C.c_double), ("done_s", C.c_double), ("steps", C.c_uint32),
                ("pad", C.c_uint32)]


class lp_server_stats(C.Structure):
    _fields_ = [("steps", C.c_uint64), ("launches", C.c_uint64), ("completed", C.c_uint64),
                ("keys_done", C.c_uint64), ("peak_bytes", C.c_uint64),
                ("budget_bytes", C.c_uint64), ("in_use_bytes", C.c_uint64),
                ("engine_bytes", C.c_uint64), ("busy_s", C.c_double),
                ("batched_ms", C.c_double)]


class lp_batch_rounds(C.Structure):
    _fields_ = [("rounds", C.c_uint32), ("pad", C.c_uint32),
                ("plan_ms", C.c_float * 12), ("task_ms", C.c_float * 12),
                ("tasks", C.c_uint64 * 12)]


def _rounds_dict(r):
    k = r.rounds
    return [{"plan_ms": r.plan_ms[i], "task_ms": r.task_ms[i], "tasks": int(r.tasks[i])}
            for i in range(k)]


_SIGS = {
    "lp_ctx_create": (_i, [C.POINTER(_p), _i]),
    "lp_ctx_destroy": (_i, [_p]),
    "lp_ctx_last_error": (C.c_char_p, [_p]),
    "lp_ctx_aux_bytes": (_u64, [_p]),
    "lp_ctx_last_launches": (_u64, [_p]),
    "lp_ctx_grid": (_u32, [_p]),
    "lp_ctx_set_timing": (_i, [_p, _i]),
    "lp_ctx_level_stats": (_i, [_p, _pu64, C.POINTER(C.c_float), C.POINTER(_i)]),
    "lp_ctx_kernel_ms": (_i, [_p, C.POINTER(C.c_float)]),
    "lp_ctx_wait": (_i, [_p]),
    "lp_ctx_set_level_cap": (_i, [_p, _u32]),
    "lp_partition_u64": (_i, [_p, _p, _u64, _u64, _i, _u64, _p, _pu64]),
    "lp_partition_u32": (_i, [_p, _p, _u64, _u32, _i, _u64, _p, _pu64]),
    "lp_partition_kv_u64": (_i, [_p, _p, _p, _u64, _u64, _i, _u64, _p, _pu64]),
    "lp_partition_u64_async": (_i, [_p, _p, _u64, _u64, _i, _u64, _p, _p]),
    "lp_partition_u32_async": (_i, [_p, _p, _u64, _u32, _i, _u64, _p, _p]),
    "lp_partition_kv_u64_async": (_i, [_p, _p, _p, _u64, _u64, _i, _u64, _p, _p]),
    "lp_smoothed_step_u64": (_i, [_p, _p, _u64, _u64, _u64, _u64, _u64, _u64, _i, _p,
                                  _pu64, _pu64, _pu64]),
    "lp_smoothed_step_u32": (_i, [_p, _p, _u64, _u32, _u64, _u64, _u64, _u64, _i, _p,
                                  _pu64, _pu64, _pu64]),
    "lp_partition_u64_noalloc": (_i, [_p, _u64, _u64, _i, _u64, _p, _p]),
    "lp_lowspace_partition_u64": (_i, [_p, _p, _u64, _u64, _u64, _u64, _p, _pu64]),
    "lp_lowspace_partition_u32": (_i, [_p, _p, _u64, _u32, _u64, _u64, _p, _pu64]),
    "lp_partition_host_u64": (_i, [_p, _p, _u64, _u64, _u64, _p, _pu64]),
    "lp_partition_host_u32": (_i, [_p, _p, _u64, _u32, _u64, _p, _pu64]),
    "lp_lowspace_implicit_partition_u64": (_i, [_p, _p, _u64, _u64, _u64, _u64, _p, _pu64]),
    "lp_lowspace_implicit_partition_u32": (_i, [_p, _p, _u64, _u32, _u64, _u64, _p, _pu64]),
    "lp_lowspace_implicit_prefix_u64": (_i, [_p, _p, _u64, _u64, _u64, _p, _pu64]),
    "lp_lowspace_implicit_prefix_u32": (_i, [_p, _p, _u64, _u32, _u64, _p, _pu64]),
    "lp_partition_batched_u64": (_i, [_p, _p, _u32, _u64, _p, _p]),
    "lp_batch_create": (_i, [_p, _p, _u32, _u64, _p, _p, C.POINTER(_p)]),
    "lp_batch_launch": (_i, [_p, _p]),
    "lp_batch_wait": (_i, [_p, _p]),
    "lp_batch_destroy": (_i, [_p]),
    "lp_autotune_batched_u64": (_i, [_p, _p, _u32, _p, _p]),
    "lp_ctx_set_batch_tuning": (_i, [_p, _p]),
    "lp_quicksort_u64": (_i, [_p, _p, _u64, _u64, _p]),
    "lp_quicksort_u32": (_i, [_p, _p, _u64, _u64, _p]),
    "lp_quicksort_ex_u64": (_i, [_p, _p, _u64, _u64, _u32, _p]),
    "lp_quicksort_ex_u32": (_i, [_p, _p, _u64, _u64, _u32, _p]),
    "lp_ctx_sort_stats": (_i, [_p, _p]),
    "lp_ctx_last_batch_keys": (_i, [_p, _pu64]),
    "lp_batch_streamed_keys": (_i, [_p, _p, _pu64]),
    "lp_ctx_last_batch_rounds": (_i, [_p, _p]),
    "lp_batch_round_stats": (_i, [_p, _p, _p]),
    "lp_server_create": (_i, [_i, _p, C.POINTER(_p)]),
    "lp_server_destroy": (_i, [_p]),
    "lp_server_last_error": (C.c_char_p, [_p]),
    "lp_server_now": (C.c_double, [_p]),
    "lp_server_submit": (_i, [_p, _p, _pu64]),
    "lp_server_step": (_i, [_p, C.POINTER(_u32)]),
    "lp_server_poll": (_i, [_p, _p, _u32, C.POINTER(_u32)]),
    "lp_server_result": (_i, [_p, _u64, C.POINTER(_p)]),
    "lp_server_fetch": (_i, [_p, _u64, _p, _u64]),
    "lp_server_release": (_i, [_p, _u64]),
    "lp_server_get_stats": (_i, [_p, _p]),
    "lp_server_streamed_keys": (_i, [_p, _pu64, _pu64]),
    "lp_server_run": (_i, [_p, _p, _u32, _u32, _p]),
    "lp_selftest_bounded_waits": (_i, [_i, C.POINTER(_u32), C.POINTER(_u32)]),
    "lp_fill_uniform_u64": (_i, [_p, _u64, _u64, _p]),
    "lp_fill_uniform_u32": (_i, [_p, _u64, _u64, _p]),
    "lp_fill_iota_u64": (_i, [_p, _u64, _p]),
}

_lib = None


def lib():
    """Load libpartition.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "libpartition.so is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name, None)
            if f is None:
                continue
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class LPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("libpartition status %d: %s" % (status, msg))
        self.status = status


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dev_ptr(t, bits):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.element_size() * 8 != bits:
        raise TypeError("expected %d-bit elements, got %s" % (bits, t.dtype))
    if not t.is_contiguous():
        raise TypeError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr()), t.numel()


class Ctx:
    """An lp_ctx on one CUDA device (lp_ctx_create / lp_ctx_destroy)."""

    def __init__(self, device=None):
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        h = C.c_void_p()
        st = lib().lp_ctx_create(C.byref(h), self.device)
        if st != LP_OK:
            raise LPError(st, "lp_ctx_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().lp_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, st):
        if st != LP_OK:
            raise LPError(st, lib().lp_ctx_last_error(self.h).decode())
        return st

    @property
    def aux_bytes(self):
        return int(lib().lp_ctx_aux_bytes(self.h))

    def wait(self):
        """lp_ctx_wait: finish the last call and raise on a device error."""
        return self.check(lib().lp_ctx_wait(self.h))

    def sort_stats(self):
        """lp_ctx_sort_stats: what the last quicksort on this context did."""
        st = lp_sort_stats()
        self.check(lib().lp_ctx_sort_stats(self.h, C.byref(st)))
        return {f: getattr(st, f) for f, _ in lp_sort_stats._fields_}

    def last_batch_rounds(self):
        """lp_ctx_last_batch_rounds: per round of the last one-shot batch."""
        r = lp_batch_rounds()
        self.check(lib().lp_ctx_last_batch_rounds(self.h, C.byref(r)))
        return _rounds_dict(r)

    def last_batch_keys(self):
        """lp_ctx_last_batch_keys: keys streamed by the last one-shot batch."""
        k = C.c_uint64()
        self.check(lib().lp_ctx_last_batch_keys(self.h, C.byref(k)))
        return int(k.value)

    @property
    def last_launches(self):
        return int(lib().lp_ctx_last_launches(self.h))

    @property
    def grid(self):
        return int(lib().lp_ctx_grid(self.h))

    def set_timing(self, on=True):
        self.check(lib().lp_ctx_set_timing(self.h, 1 if on else 0))

    def set_level_cap(self, levels=0):
        """lp_ctx_set_level_cap: level at which LP_SMOOTHED hands an open range
        to the low-space partition (0: the last level)."""
        self.check(lib().lp_ctx_set_level_cap(self.h, int(levels)))

    def kernel_ms(self):
        """Event-timed duration of the last timed call's partition kernel (ms)."""
        v = C.c_float()
        self.check(lib().lp_ctx_kernel_ms(self.h, C.byref(v)))
        return float(v.value)

    def level_stats(self):
        """[(lo, hi, b, g, ms)] for each level of the last partition call."""
        rng = (C.c_uint64 * (4 * LP_MAX_LEVELS))()
        ms = (C.c_float * LP_MAX_LEVELS)()
        nl = C.c_int()
        self.check(lib().lp_ctx_level_stats(self.h, rng, ms, C.byref(nl)))
        return [(int(rng[4 * i]), int(rng[4 * i + 1]), int(rng[4 * i + 2]), int(rng[4 * i + 3]),
                 float(ms[i])) for i in range(nl.value)]


def lp_ctx_create(device=None):
    return Ctx(device)


def lp_partition_u64(ctx, keys, pivot, variant=LP_SMOOTHED, seed=0, stream=None):
    p, n = _dev_ptr(keys, 64)
    t = C.c_uint64()
    ctx.check(lib().lp_partition_u64(ctx.h, p, n, int(pivot), int(variant), int(seed),
                                     _stream(stream), C.byref(t)))
    return int(t.value)


def lp_partition_u32(ctx, keys, pivot, variant=LP_SMOOTHED, seed=0, stream=None):
    p, n = _dev_ptr(keys, 32)
    t = C.c_uint64()
    ctx.check(lib().lp_partition_u32(ctx.h, p, n, int(pivot), int(variant), int(seed),
                                     _stream(stream), C.byref(t)))
    return int(t.value)


def lp_partition_kv_u64(ctx, keys, vals, pivot, variant=LP_SMOOTHED, seed=0, stream=None):
    p, n = _dev_ptr(keys, 64)
    q, m = _dev_ptr(vals, 64)
    if m != n:
        raise ValueError("keys and vals differ in length")
    t = C.c_uint64()
    ctx.check(lib().lp_partition_kv_u64(ctx.h, p, q, n, int(pivot), int(variant), int(seed),
                                        _stream(stream), C.byref(t)))
    return int(t.value)


def lp_partition_u64_async(ctx, keys, pivot, d_split, variant=LP_SMOOTHED, seed=0, stream=None):
    p, n = _dev_ptr(keys, 64)
    s, _ = _dev_ptr(d_split, 64)
    return ctx.check(lib().lp_partition_u64_async(ctx.h, p, n, int(pivot), int(variant),
                                                  int(seed), _stream(stream), s))


def lp_partition_u32_async(ctx, keys, pivot, d_split, variant=LP_SMOOTHED, seed=0, stream=None):
    p, n = _dev_ptr(keys, 32)
    s, _ = _dev_ptr(d_split, 64)
    return ctx.check(lib().lp_partition_u32_async(ctx.h, p, n, int(pivot), int(variant),
                                                  int(seed), _stream(stream), s))


def lp_partition_kv_u64_async(ctx, keys, vals, pivot, d_split, variant=LP_SMOOTHED, seed=0,
                              stream=None):
    p, n = _dev_ptr(keys, 64)
    q, _ = _dev_ptr(vals, 64)
    s, _ = _dev_ptr(d_split, 64)
    return ctx.check(lib().lp_partition_kv_u64_async(ctx.h, p, q, n, int(pivot), int(variant),
                                                     int(seed), _stream(stream), s))


def lp_partition_u64_noalloc(keys, pivot, d_split, variant=LP_SMOOTHED, seed=0, stream=None):
    """Allocation-free partition (no lp_ctx): t is written to d_split on the device.
    For callers that cannot allocate device memory; see libpartition.h."""
    p, n = _dev_ptr(keys, 64)
    s, _ = _dev_ptr(d_split, 64)
    st = lib().lp_partition_u64_noalloc(p, n, int(pivot), int(variant), int(seed),
                                        _stream(stream), s)
    if st != LP_OK:
        raise LPError(st, "lp_partition_u64_noalloc")


def _segments(views, pivots):
    arr = (lp_segment_u64 * len(views))()
    for s, (v, p) in enumerate(zip(views, pivots)):
        ptr, n = _dev_ptr(v, 64)
        arr[s].keys = ptr.value if n else None
        arr[s].n = n
        arr[s].pivot = int(p)
    return arr


def lp_partition_batched_u64(ctx, views, pivots, d_splits, seed=0, stream=None):
    """Partition every tensor in `views` (uint64 keys, non-overlapping) by its
    pivot in one persistent launch; splits go to d_splits (device int64)."""
    segs = _segments(views, pivots)
    sp, m = _dev_ptr(d_splits, 64)
    if m < len(views):
        raise ValueError("d_splits too short")
    ctx.check(lib().lp_partition_batched_u64(ctx.h, segs, len(views), int(seed),
                                             _stream(stream), sp))


class Batch:
    """lp_batch: a segment list captured once into a CUDA graph, replayed."""

    def __init__(self, ctx, views, pivots, d_splits, seed=0, stream=None):
        self.ctx = ctx
        self._segs = _segments(views, pivots)
        sp, _ = _dev_ptr(d_splits, 64)
        h = C.c_void_p()
        ctx.check(lib().lp_batch_create(ctx.h, self._segs, len(views), int(seed), sp,
                                        _stream(stream), C.byref(h)))
        self.h = h

    def launch(self, stream=None):
        self.ctx.check(lib().lp_batch_launch(self.h, _stream(stream)))

    def wait(self, stream=None):
        """lp_batch_wait: finish the last launch and raise on a device error."""
        return self.ctx.check(lib().lp_batch_wait(self.h, _stream(stream)))

    def round_stats(self, stream=None):
        """lp_batch_round_stats: per round of the last launch."""
        r = lp_batch_rounds()
        self.ctx.check(lib().lp_batch_round_stats(self.h, _stream(stream), C.byref(r)))
        return _rounds_dict(r)

    def streamed_keys(self, stream=None):
        """lp_batch_streamed_keys: keys streamed by the last launch."""
        k = C.c_uint64()
        self.ctx.check(lib().lp_batch_streamed_keys(self.h, _stream(stream), C.byref(k)))
        return int(k.value)

    def close(self):
        if getattr(self, "h", None):
            lib().lp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lp_autotune_batched_u64(ctx, sizes, stream=None):
    arr = (C.c_uint64 * len(sizes))(*[int(x) for x in sizes])
    best = lp_batch_tuning()
    ctx.check(lib().lp_autotune_batched_u64(ctx.h, arr, len(sizes), _stream(stream),
                                            C.byref(best)))
    return {"ctas": best.ctas, "line_bytes": best.line_bytes, "min_chunks": best.min_chunks,
            "group_workers": best.group_workers, "min_chunks_residual": best.min_chunks_residual,
            "onchip_slices": best.onchip_slices}


def lp_ctx_set_batch_tuning(ctx, ctas=0, line_bytes=0, min_chunks=0, group_workers=0,
                            min_chunks_residual=0, onchip_slices=0):
    t = lp_batch_tuning(ctas, line_bytes, min_chunks, group_workers, min_chunks_residual,
                        onchip_slices)
    ctx.check(lib().lp_ctx_set_batch_tuning(ctx.h, C.byref(t)))


def lp_quicksort(ctx, keys, seed=0, stream=None, pivot_samples=3):
    """Sort a uint64 or uint32 device tensor ascending in place; each pivot is
    the median of pivot_samples (3 or 15) seeded keys."""
    bits = keys.element_size() * 8
    p, n = _dev_ptr(keys, bits)
    if pivot_samples == 3:
        f = lib().lp_quicksort_u64 if bits == 64 else lib().lp_quicksort_u32
        ctx.check(f(ctx.h, p, n, int(seed), _stream(stream)))
    else:
        f = lib().lp_quicksort_ex_u64 if bits == 64 else lib().lp_quicksort_ex_u32
        ctx.check(f(ctx.h, p, n, int(seed), int(pivot_samples), _stream(stream)))


def lp_lowspace_partition(ctx, keys, pivot, B=4096, base_keys=0, stream=None):
    """Blocked-Prefix-Sum partition with block size B; returns the split t."""
    bits = keys.element_size() * 8
    p, n = _dev_ptr(keys, bits)
    f = lib().lp_lowspace_partition_u64 if bits == 64 else lib().lp_lowspace_partition_u32
    t = C.c_uint64()
    ctx.check(f(ctx.h, p, n, int(pivot), int(B), int(base_keys), _stream(stream), C.byref(t)))
    return int(t.value)


def lp_partition_host(ctx, keys, pivot, seed=0, stream=None):
    """Partition a CPU tensor (int64 / int32 holding uint64 / uint32 keys) in
    place through lp_partition_host_*; pinned memory lets the copies overlap.
    Returns the split t."""
    if not isinstance(keys, torch.Tensor) or keys.is_cuda:
        raise TypeError("expected a CPU tensor")
    if not keys.is_contiguous():
        raise TypeError("expected a contiguous tensor")
    bits = keys.element_size() * 8
    if bits not in (32, 64):
        raise TypeError("expected 32- or 64-bit keys")
    f = lib().lp_partition_host_u64 if bits == 64 else lib().lp_partition_host_u32
    t = C.c_uint64()
    ctx.check(f(ctx.h, C.c_void_p(keys.data_ptr()), keys.numel(), int(pivot), int(seed),
                _stream(stream), C.byref(t)))
    return int(t.value)


def lp_lowspace_implicit_partition(ctx, keys, pivot, B=4096, base_keys=0, stream=None):
    """Blocked-Prefix-Sum partition with the block values kept in key order
    (B = 0: the paper's 4 * ceil(log2(n + 1)) + 2); returns the split t."""
    bits = keys.element_size() * 8
    p, n = _dev_ptr(keys, bits)
    f = (lib().lp_lowspace_implicit_partition_u64 if bits == 64
         else lib().lp_lowspace_implicit_partition_u32)
    t = C.c_uint64()
    ctx.check(f(ctx.h, p, n, int(pivot), int(B), int(base_keys), _stream(stream), C.byref(t)))
    return int(t.value)


def lp_lowspace_implicit_prefix(ctx, keys, pivot, B=4096, stream=None):
    """The first three phases of the above (keys left with the values
    encoded); returns t."""
    bits = keys.element_size() * 8
    p, n = _dev_ptr(keys, bits)
    f = (lib().lp_lowspace_implicit_prefix_u64 if bits == 64
         else lib().lp_lowspace_implicit_prefix_u32)
    t = C.c_uint64()
    ctx.check(f(ctx.h, p, n, int(pivot), int(B), _stream(stream), C.byref(t)))
    return int(t.value)


def lp_smoothed_step(ctx, keys, pivot, b, g, seed=0, level=0, strided=False, stream=None):
    """One Partial Partition Step; returns (vmin, vmax, count)."""
    bits = keys.element_size() * 8
    p, n = _dev_ptr(keys, bits)
    f = lib().lp_smoothed_step_u64 if bits == 64 else lib().lp_smoothed_step_u32
    vmin, vmax, cnt = C.c_uint64(), C.c_uint64(), C.c_uint64()
    ctx.check(f(ctx.h, p, n, int(pivot), int(b), int(g), int(seed), int(level),
                1 if strided else 0, _stream(stream), C.byref(vmin), C.byref(vmax),
                C.byref(cnt)))
    return int(vmin.value), int(vmax.value), int(cnt.value)


def lp_fill_uniform_u64(keys, seed, stream=None):
    p, n = _dev_ptr(keys, 64)
    st = lib().lp_fill_uniform_u64(p, n, int(seed), _stream(stream))
    if st != LP_OK:
        raise LPError(st, "lp_fill_uniform_u64")


def lp_fill_uniform_u32(keys, seed, stream=None):
    p, n = _dev_ptr(keys, 32)
    st = lib().lp_fill_uniform_u32(p, n, int(seed), _stream(stream))
    if st != LP_OK:
        raise LPError(st, "lp_fill_uniform_u32")


def lp_fill_iota_u64(vals, stream=None):
    p, n = _dev_ptr(vals, 64)
    st = lib().lp_fill_iota_u64(p, n, _stream(stream))
    if st != LP_OK:
        raise LPError(st, "lp_fill_iota_u64")


# ---------------------------------------------------------------- serving

LP_REQ_PARTITION = 0
LP_REQ_SORT = 1
LP_SERVE_CONTINUOUS = 0
LP_SERVE_ONE_AT_A_TIME = 1


def _completion_dict(c):
    return {f: getattr(c, f) for f, _ in lp_completion._fields_ if f != "pad"}


class Server:
    """lp_server: continuous-batching engine for partition and sort requests."""

    def __init__(self, device=None, budget_bytes=1 << 30, max_slots=0, max_segments=0, seed=1,
                 keep_results=False, timing=False):
        if device is None:
            device = torch.cuda.current_device()
        cfg = lp_server_config(int(budget_bytes), int(max_slots), int(max_segments), int(seed),
                               1 if keep_results else 0, 1 if timing else 0)
        h = C.c_void_p()
        st = lib().lp_server_create(int(device), C.byref(cfg), C.byref(h))
        if st != LP_OK:
            raise LPError(st, "lp_server_create")
        self.h = h

    def check(self, st):
        if st != LP_OK:
            raise LPError(st, lib().lp_server_last_error(self.h).decode())
        return st

    @staticmethod
    def request(kind, key_bits, n, pivot=0, seed=0, src=None, arrival_s=0.0):
        r = lp_request()
        r.kind, r.key_bits, r.n, r.pivot, r.seed = int(kind), int(key_bits), int(n), \
            int(pivot), int(seed)
        if src is not None:
            p, m = _dev_ptr(src, int(key_bits))
            if m != n:
                raise ValueError("src length differs from n")
            r.d_src = p.value
        r.arrival_s = float(arrival_s)
        return r

    def now(self):
        return float(lib().lp_server_now(self.h))

    def submit(self, kind, key_bits, n, pivot=0, seed=0, src=None, arrival_s=None):
        r = self.request(kind, key_bits, n, pivot, seed, src,
                         self.now() if arrival_s is None else arrival_s)
        i = C.c_uint64()
        self.check(lib().lp_server_submit(self.h, C.byref(r), C.byref(i)))
        return int(i.value)

    def step(self):
        k = C.c_uint32()
        self.check(lib().lp_server_step(self.h, C.byref(k)))
        return int(k.value)

    def poll(self, cap=1024):
        buf = (lp_completion * cap)()
        got = C.c_uint32()
        self.check(lib().lp_server_poll(self.h, buf, cap, C.byref(got)))
        return [_completion_dict(buf[i]) for i in range(got.value)]

    def result_ptr(self, id_):
        p = C.c_void_p()
        self.check(lib().lp_server_result(self.h, int(id_), C.byref(p)))
        return int(p.value)

    def fetch(self, id_, n, key_bits):
        """The finished request's keys as a numpy array (keep_results)."""
        import numpy as np
        out = np.empty(int(n), dtype=np.uint64 if key_bits == 64 else np.uint32)
        self.check(lib().lp_server_fetch(self.h, int(id_), C.c_void_p(out.ctypes.data),
                                         out.nbytes))
        return out

    def release(self, id_):
        self.check(lib().lp_server_release(self.h, int(id_)))

    def stats(self):
        st = lp_server_stats()
        self.check(lib().lp_server_get_stats(self.h, C.byref(st)))
        return {f: getattr(st, f) for f, _ in lp_server_stats._fields_}

    def streamed_keys(self):
        """(uint64 keys, uint32 keys) streamed by the engine's batched launches."""
        a, b = C.c_uint64(), C.c_uint64()
        self.check(lib().lp_server_streamed_keys(self.h, C.byref(a), C.byref(b)))
        return int(a.value), int(b.value)

    def run(self, requests, mode=LP_SERVE_CONTINUOUS):
        """Open-loop run of lp_request records (arrival_s relative to the start)."""
        arr = (lp_request * len(requests))(*requests)
        out = (lp_completion * len(requests))()
        self.check(lib().lp_server_run(self.h, arr, len(requests), int(mode), out))
        return [_completion_dict(out[i]) for i in range(len(requests))]

    def close(self):
        if getattr(self, "h", None):
            lib().lp_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lp_selftest_bounded_waits(device=0):
    """(mbarrier wait gave up, grid barrier gave up): both 1 on a working build."""
    a, b = C.c_uint32(), C.c_uint32()
    st = lib().lp_selftest_bounded_waits(int(device), C.byref(a), C.byref(b))
    if st != LP_OK:
        raise LPError(st, "lp_selftest_bounded_waits")
    return int(a.value), int(b.value)
