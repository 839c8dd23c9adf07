"""Seeded synthetic inputs for partition and sort workloads.

This module holds the input generators only -- none of the partition
arithmetic.  Both the CPU oracle side and the CUDA side of the tests, and the
benchmark, draw their inputs from here, so that the two sides see identical
arrays.

Keys follow the paper's experimental setup (Sec. 5): each key is drawn
independently and uniformly, so each is "randomly larger or smaller than the
pivot"; sort inputs add already-sorted, reverse-sorted and heavy-duplicate
variants.  The generator is SplitMix64 (Steele, Lea, Flood 2014): key i is the
i-th output of the generator whose state starts at `seed`.  The library's
device-side filler (lp_fill_uniform_u64 / _u32) produces the same values.
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix_outputs(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start..start+count-1 of SplitMix64 seeded with `seed` (uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
        z = np.uint64(seed & (2**64 - 1)) + k * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform_u64(n: int, seed: int) -> np.ndarray:
    """n keys uniform over [0, 2^64)."""
    out = np.empty(n, dtype=np.uint64)
    step = 1 << 24
    for s in range(0, n, step):
        c = min(step, n - s)
        out[s:s + c] = splitmix_outputs(seed, s, c)
    return out


def uniform_u32(n: int, seed: int) -> np.ndarray:
    """n keys uniform over [0, 2^32): the low 32 bits of the 64-bit stream."""
    return (uniform_u64(n, seed) & np.uint64(0xFFFFFFFF)).astype(np.uint32)


def heavy_duplicates_u64(n: int, seed: int, distinct: int = 16) -> np.ndarray:
    """n keys uniform over [0, distinct)."""
    return uniform_u64(n, seed) % np.uint64(distinct)


def sorted_u64(n: int, seed: int) -> np.ndarray:
    return np.sort(uniform_u64(n, seed))


def reverse_sorted_u64(n: int, seed: int) -> np.ndarray:
    return np.sort(uniform_u64(n, seed))[::-1].copy()


def quantile_pivot(num: int, den: int, bits: int = 64) -> int:
    """Pivot p with [x <= p] selecting the fraction num/den of a uniform key
    range [0, 2^bits): p = ceil(num * 2^bits / den) - 1, in exact integers."""
    top = num << bits
    p = -(-top // den) - 1
    return max(0, min(p, (1 << bits) - 1))


def log_uniform_sizes(count: int, seed: int, lo_log2: int, hi_log2: int) -> np.ndarray:
    """count sizes floor(2^(lo + (hi-lo)*u)), u uniform in [0,1) from the stream."""
    u = splitmix_outputs(seed, 0, count).astype(np.float64) / float(2**64)
    return np.floor(np.exp2(lo_log2 + (hi_log2 - lo_log2) * u)).astype(np.int64)
