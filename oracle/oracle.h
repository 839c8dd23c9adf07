/*
 * oracle.h -- plain serial CPU oracle for in-place parallel partition
 * (Kuszmaul & Westover, "In-Place Parallel-Partition Algorithms using
 * Exclusive-Read-and-Write Memory", arXiv 2004.12532).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code with the CUDA library (no common headers, helpers or generators).
 *
 * Conventions (readings of the paper, see the "Readings" list in the design
 * notes):
 *   - arrays are 0-indexed; the paper is 1-indexed (Sec. 2, problem statement);
 *   - the decider is dec(x) = [x <= pivot]: a key <= pivot is a predecessor,
 *     a key > pivot a successor (Fig. "Smoothed Striding Algorithm", the
 *     comparison A[low] <= pivotValue);
 *   - every partition returns the split t = number of predecessors, so that
 *     a[0..t) are predecessors and a[t..n) successors.
 * All arithmetic is integer; nothing here is floating point.
 */
#ifndef PARTITION_ORACLE_H
#define PARTITION_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* --- counter-based random source (SplitMix64, Steele/Lea/Flood 2014) --- */
/* k-th output (k >= 0) of the SplitMix64 generator whose state starts at seed. */
uint64_t or_stream(uint64_t seed, uint64_t k);
/* floor(r * g / 2^64): maps a uniform 64-bit word onto {0..g-1}. */
uint64_t or_range(uint64_t r, uint64_t g);

/* --- the problem (Sec. 2, "The Parallel Partition Problem") --- */
uint64_t or_count_u64(const uint64_t *a, uint64_t n, uint64_t pivot);
uint64_t or_count_u32(const uint32_t *a, uint64_t n, uint32_t pivot);
/* Serial in-place two-pointer (Hoare) partition; returns t. */
uint64_t or_partition_u64(uint64_t *a, uint64_t n, uint64_t pivot);
uint64_t or_partition_u32(uint32_t *a, uint64_t n, uint32_t pivot);
/* Same, moving payload v[i] together with key a[i]. */
uint64_t or_partition_kv_u64(uint64_t *a, uint64_t *v, uint64_t n, uint64_t pivot);
/* Partition each of `rows` independent rows of length len (row-major). */
void or_partition_rows_u64(uint64_t *a, uint64_t rows, uint64_t len,
                           uint64_t pivot, uint64_t *t_out);

/* --- Smoothed Striding (Sec. 4) --- */
/* Draw X[0..s) for level `level` of a run seeded with `seed` (Sec. 4,
 * "Set each of X[1..s] to be uniformly random ... in {1..g}"). */
void or_draw_X(uint64_t seed, uint64_t level, uint64_t s, uint64_t g, uint64_t *X);
/* Geometry of a step on a range of n keys with lines of b keys and g groups:
 * L = ceil(n/b) lines, s = ceil(L/g) chunks. */
uint64_t or_num_chunks(uint64_t n, uint64_t b, uint64_t g);
/* The Partial Partition Step on a[0..n): group i holds, for every chunk j,
 * line j*g + (X[j]+i) mod g (lines past the end are virtual and skipped).
 * Each group is partitioned serially in its own slot order.  Outputs:
 * k[i] predecessors of group i, v[i] the index of group i's first successor
 * slot (one past its last slot when it has none), vmin/vmax over the non-empty
 * groups.  k and v may be NULL.  Returns 0, or -1 on bad arguments. */
int or_smoothed_step_u64(uint64_t *a, uint64_t n, uint64_t pivot, uint64_t b,
                         uint64_t g, const uint64_t *X, uint64_t *k, uint64_t *v,
                         uint64_t *vmin, uint64_t *vmax);
int or_smoothed_step_u32(uint32_t *a, uint64_t n, uint32_t pivot, uint64_t b,
                         uint64_t g, const uint64_t *X, uint64_t *k, uint64_t *v,
                         uint64_t *vmin, uint64_t *vmax);
/* Recursive Smoothed Striding: partial steps on the residual [vmin, vmax)
 * with fresh X per level until the residual has at most `base` keys, then a
 * serial partition.  Line size b; g = min(gmax, ceil(n/(b*smin))), at least 2.
 * Returns t.  Writes the number of levels run to *levels (may be NULL). */
uint64_t or_smoothed_partition_u64(uint64_t *a, uint64_t n, uint64_t pivot,
                                   uint64_t seed, uint64_t b, uint64_t gmax,
                                   uint64_t smin, uint64_t base, uint64_t *levels);
/* Strided Algorithm (Francis-Pannan, Sec. 4): the step with X == 0 followed by
 * a serial cleanup of [vmin, vmax).  Returns t. */
uint64_t or_strided_partition_u64(uint64_t *a, uint64_t n, uint64_t pivot,
                                  uint64_t b, uint64_t g);

/* --- Blocked-Prefix-Sum partition (Sec. 3), explicit prefix counters --- */
/* The decider used by the low-space routines: flip == 0 -> [x <= pivot];
 * flip == 1 -> [x > pivot] on the logically reversed array (Fig. main
 * functions, ParallelPartition's role swap). */
void or_make_successor_heavy_u64(uint64_t *a, uint64_t n, uint64_t pivot, int flip);
/* v[i] = predecessors in blocks 0..i; blocks of B keys, the last block takes
 * the remainder (size B..2B-1).  Returns the number of blocks floor(n/B). */
uint64_t or_block_prefix_u64(const uint64_t *a, uint64_t n, uint64_t pivot, int flip,
                             uint64_t B, uint64_t *v);
/* In-place reordering (Lemma "Reordering phase"): needs successor-heavy
 * prefixes and v from or_block_prefix_u64. */
void or_reorder_u64(uint64_t *a, uint64_t n, uint64_t pivot, int flip, uint64_t B,
                    const uint64_t *v);
/* Full low-space partition: count, role swap, preprocessing, prefix, reorder.
 * Returns t. */
uint64_t or_lowspace_partition_u64(uint64_t *a, uint64_t n, uint64_t pivot, uint64_t B);

/* --- Blocked-Prefix-Sum partition, values kept in key order (Sec. 3,
 * Lemma bitstore2; parity pinned by the round trip, brute-force prefixes
 * and the partition postcondition) --- */
/* L = ceil(log2(n + 1)), the bits of a value in [0, n]. */
uint64_t or_bits_for(uint64_t n);
/* Encode v (< 2^L) in x[0 .. 4L+2); first = 1 on the first call for x. */
void or_bitstore_encode_u64(uint64_t *x, uint64_t L, uint64_t v, int first);
/* Decode the value of x[0 .. 4L+2); restore = 1 puts back overwritten keys. */
uint64_t or_bitstore_decode_u64(uint64_t *x, uint64_t L, int restore);
/* Count, role swap, MakeSuccessorHeavy, then the prefix phase with block i
 * encoding the predecessors before it (blocks of B >= 4L + 2 keys, the last
 * taking the remainder).  Returns t; *flip gets the role (may be NULL). */
uint64_t or_implicit_prefix_u64(uint64_t *a, uint64_t n, uint64_t pivot, uint64_t B, int *flip);
/* The whole fully in-place partition.  Returns t. */
uint64_t or_implicit_partition_u64(uint64_t *a, uint64_t n, uint64_t pivot, uint64_t B);

/* --- quicksort on the partition (Sec. 5, "A Full Quicksort") --- */
void or_quicksort_u64(uint64_t *a, uint64_t n, uint64_t seed);
void or_quicksort_u32(uint32_t *a, uint64_t n, uint64_t seed);

#ifdef __cplusplus
}
#endif
#endif
