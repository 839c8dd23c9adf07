/*
 * libpartition -- in-place parallel partition on one GB300 GPU (sm_103a).
 *
 * Implements the algorithms of Kuszmaul & Westover, "In-Place
 * Parallel-Partition Algorithms using Exclusive-Read-and-Write Memory"
 * (arXiv 2004.12532): the Smoothed Striding Algorithm (Sec. 4), the Strided
 * Algorithm it builds on (Sec. 4, after Francis & Pannan), the
 * Blocked-Prefix-Sum ("low-space") partition (Sec. 3), and a quicksort built on
 * the partition (Sec. 5, "A Full Quicksort").
 *
 * The problem (Sec. 2, "The Parallel Partition Problem"): reorder an array so
 * that every predecessor precedes every successor.  Here the decider is
 * dec(x) = [x <= pivot]: keys <= pivot are predecessors.  Arrays are
 * 0-indexed; every partition reports the split t = number of predecessors, so
 * keys[0..t) <= pivot < keys[t..n) afterwards, and the array is a permutation
 * of its input.  The order inside each side is unspecified but deterministic
 * for a given input, seed and device.
 *
 * Conventions for every call:
 *   - key / value pointers are DEVICE pointers owned by the caller; the library
 *     reorders them in place and never frees or reallocates them.  They must be
 *     naturally aligned (8 bytes for uint64_t, 4 for uint32_t); 16-byte
 *     alignment is not required.
 *   - work is enqueued on the caller's cudaStream_t and is stream-ordered.
 *     Calls that take a host `*_out` pointer synchronise that stream before
 *     returning; `_async` calls do not.
 *   - scratch memory belongs to the lp_ctx (allocated once at creation, a few
 *     KB plus what a call needs, never more than 1% of the array's bytes for
 *     the partition calls); lp_ctx_aux_bytes reports it.  Calls that share an
 *     lp_ctx share its scratch: issue them on one stream, or synchronise
 *     between them.
 *   - every call returns an lp_status and never aborts the process; on error
 *     lp_ctx_last_error() describes it.  On LP_ERR_TIMEOUT or LP_ERR_INTERNAL
 *     the array is a permutation of its input but may not be partitioned.
 *   - n == 0 is valid and returns t = 0; a null key pointer with n > 0 is
 *     LP_ERR_INVALID_ARG.
 */
#ifndef LIBPARTITION_H
#define LIBPARTITION_H

#include <stdint.h>
#include <cuda_runtime.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LP_OK = 0,
  LP_ERR_INVALID_ARG = 1, /* null pointer, bad size, bad variant, ... */
  LP_ERR_MISALIGNED = 2,  /* only from calls that require 16-byte aligned input */
  LP_ERR_OOM = 3,         /* a scratch allocation failed */
  LP_ERR_BUDGET = 4,      /* the server's memory budget cannot hold a request */
  LP_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  LP_ERR_CUDA = 6,        /* a CUDA runtime call failed; see lp_ctx_last_error */
  LP_ERR_INTERNAL = 7     /* a device-side consistency check failed */
} lp_status;

typedef enum {
  LP_SMOOTHED = 0, /* Recursive Smoothed Striding (Sec. 4); a range the recursion
                      fails to shrink goes to LP_LOWSPACE (lp_ctx_set_level_cap) */
  LP_STRIDED = 1,  /* Strided Algorithm: the step with X == 0, then the open
                      range [v_min, v_max) by LP_LOWSPACE (the paper's cleanup is
                      serial) */
  LP_LOWSPACE = 2, /* Blocked-Prefix-Sum partition (Sec. 3), explicit prefix */
  LP_HYBRID = 3    /* Hybrid Smoothed Striding (Theorem 4.3): one step with
                      random X, the open range by LP_LOWSPACE */
} lp_variant;

typedef struct lp_ctx lp_ctx;

/* Creates a context on CUDA device `device` (which becomes current for the
 * calling thread).  Queries the SM count and allocates the fixed scratch. */
lp_status lp_ctx_create(lp_ctx **ctx, int device);
/* Frees the context's scratch.  Outstanding work must have completed. */
lp_status lp_ctx_destroy(lp_ctx *ctx);
/* Message of the last error on this context ("" when none).  Owned by ctx. */
const char *lp_ctx_last_error(const lp_ctx *ctx);
/* Device scratch bytes held by the context (fixed part + the largest
 * per-call part so far). */
uint64_t lp_ctx_aux_bytes(const lp_ctx *ctx);
/* Kernel launches made by the last call on this context. */
uint64_t lp_ctx_last_launches(const lp_ctx *ctx);
/* Number of CTAs the streaming kernels use per launch on this device. */
uint32_t lp_ctx_grid(const lp_ctx *ctx);

/* Level records of a Smoothed / Strided partition (lp_ctx_level_stats). */
#define LP_MAX_LEVELS 10
/* Residual-shrink guard of LP_SMOOTHED (the Hybrid scheme of Sec. 4, Theorem
 * 4.3, as a fallback): the recursion hands the range it has left open to the
 * Blocked-Prefix-Sum partition (LP_LOWSPACE, B = 4096) once two levels, each
 * with fresh offsets X, have each left at least 7/8 of the range before them
 * open, or when a range is still open at level `levels` (1 .. LP_MAX_LEVELS - 1;
 * 0 restores the default, LP_MAX_LEVELS - 1).  The result is the same
 * partition (split and sides) whichever path finishes it; a small cap forces
 * the handoff, which is how tests reach it.  Applies to later LP_SMOOTHED
 * calls on ctx with arrays too large to finish on chip at once; those calls
 * hold the low-space counters (8 bytes per 4096 keys) in ctx.
 * LP_ERR_INVALID_ARG for levels >= LP_MAX_LEVELS. */
lp_status lp_ctx_set_level_cap(lp_ctx *ctx, uint32_t levels);
/* enable != 0: later partition calls on ctx record a CUDA event on their
 * stream before each partial-step kernel and after the last one. */
lp_status lp_ctx_set_timing(lp_ctx *ctx, int enable);
/* Waits for the last call issued on ctx (on that call's stream) and returns
 * its device status: LP_OK, LP_ERR_TIMEOUT (a bounded device wait gave up) or
 * LP_ERR_INTERNAL.  This is how the outcome of the _async partitions and of
 * lp_partition_batched_u64 is learnt. */
lp_status lp_ctx_wait(lp_ctx *ctx);
/* Level structure of the last Smoothed / Strided partition call on ctx (the
 * recursion of Sec. 4 on [v_min, v_max)): for level L < LP_MAX_LEVELS,
 * ranges[4L..4L+3] = {lo, hi, b, g} of the range that level partitioned
 * (all zero for a level that had nothing left to do; g == 0 marks the on-chip
 * base case, g == UINT64_MAX a range handed to the low-space partition by the
 * residual-shrink guard), and ms[L] = the level's duration in milliseconds from device
 * timestamps (ms may be NULL).  After an LP_LOWSPACE call (or
 * lp_lowspace_partition_*) the entries are its phases instead: ms[0..4] =
 * count, MakeSuccessorHeavy, block prefix, innermost prefix on chip, Reorder,
 * with all ranges zero.  Synchronises the last call's stream.
 * *levels receives LP_MAX_LEVELS. */
lp_status lp_ctx_level_stats(lp_ctx *ctx, uint64_t *ranges, float *ms, int *levels);
/* Duration in milliseconds, from CUDA events on the call's stream, of the
 * partition kernel of the last call on ctx (timing must have been enabled for
 * that call).  Synchronises on the end event. */
lp_status lp_ctx_kernel_ms(lp_ctx *ctx, float *ms);

/* ---------------------------------------------------------------- partition
 * Partition keys[0..n) by [x <= pivot] (Sec. 2).  `variant` selects the
 * algorithm; `seed` drives the random offsets X of Smoothed Striding (Sec. 4,
 * "Set each of X[1..s] to be uniformly random") and is ignored by variants
 * without randomness.  *split_out (host) receives t; the call synchronises
 * `stream`.  */
lp_status lp_partition_u64(lp_ctx *ctx, uint64_t *keys, uint64_t n, uint64_t pivot,
                           lp_variant variant, uint64_t seed, cudaStream_t stream,
                           uint64_t *split_out);
lp_status lp_partition_u32(lp_ctx *ctx, uint32_t *keys, uint64_t n, uint32_t pivot,
                           lp_variant variant, uint64_t seed, cudaStream_t stream,
                           uint64_t *split_out);
/* Key + payload: vals[i] moves with keys[i].  Two separate arrays of n
 * entries (structure of arrays). */
lp_status lp_partition_kv_u64(lp_ctx *ctx, uint64_t *keys, uint64_t *vals, uint64_t n,
                              uint64_t pivot, lp_variant variant, uint64_t seed,
                              cudaStream_t stream, uint64_t *split_out);
/* As above without synchronising: t is written to the device word *d_split
 * when the stream reaches the end of the call (UINT64_MAX, never a valid
 * split, after a device-side failure; lp_ctx_wait reports which).  An LP_SMOOTHED
 * call on an array too large to finish on chip may first grow ctx's scratch
 * (the residual-shrink guard's counters), which synchronises `stream` once. */
lp_status lp_partition_u64_async(lp_ctx *ctx, uint64_t *keys, uint64_t n, uint64_t pivot,
                                 lp_variant variant, uint64_t seed, cudaStream_t stream,
                                 uint64_t *d_split);
lp_status lp_partition_u32_async(lp_ctx *ctx, uint32_t *keys, uint64_t n, uint32_t pivot,
                                 lp_variant variant, uint64_t seed, cudaStream_t stream,
                                 uint64_t *d_split);
lp_status lp_partition_kv_u64_async(lp_ctx *ctx, uint64_t *keys, uint64_t *vals,
                                    uint64_t n, uint64_t pivot, lp_variant variant,
                                    uint64_t seed, cudaStream_t stream, uint64_t *d_split);

/* ------------------------------------------------------ batched partition
 * Many independent partitions in one persistent cooperative launch: segment
 * s is keys[0..n) of segs[s], partitioned by [x <= pivot] with the Recursive
 * Smoothed Striding scheme (a step per round on its open range, the range
 * finished on chip once one CTA, or the shared memory of at most the launch's
 * CTAs, can hold it).  Per segment the result is a partition with split t_s
 * written to d_splits[s] (device, count entries), deterministic for a given
 * batch, seed and tuning.  Segments must not overlap.  Scratch: about 144
 * bytes per segment record plus 28 bytes per segment of plan space and 64 KB
 * of slice counts, held by ctx. */
typedef struct {
  uint64_t *keys; /* device pointer, naturally aligned */
  uint64_t n;
  uint64_t pivot;
} lp_segment_u64;

/* Knobs of the batched engine (0 = default); lp_autotune_batched_u64 picks
 * them. */
typedef struct {
  uint32_t ctas;          /* CTAs of the persistent launch (<= lp_ctx_grid) */
  uint32_t line_bytes;    /* line size b * key bytes of the steps: 128 .. 2048 */
  uint32_t min_chunks;    /* lines per group, at least */
  uint32_t group_workers; /* groups per segment step, at most */
  uint32_t min_chunks_residual; /* lines per group, at least, in steps after the first */
  uint32_t onchip_slices; /* a range finished on chip by several CTAs spans at most this
                             many CTAs' shared memory (0 = the launch's grid); below the
                             grid it also shortens the windows their counts share */
} lp_batch_tuning;

/* One-shot: copies the segment list (host) to the device and runs the batch on
 * `stream` (asynchronous).  Uses the tuning stored in ctx. */
lp_status lp_partition_batched_u64(lp_ctx *ctx, const lp_segment_u64 *segs, uint32_t count,
                                   uint64_t seed, cudaStream_t stream, uint64_t *d_splits);

/* A reusable batch: the segment list is uploaded once and the whole batch
 * (set-up kernel, resets, persistent launch) is captured into a CUDA graph
 * that lp_batch_launch replays -- one graph launch per batch, on any stream.
 * The capture uses a stream of the library's own; `stream` is unused.  The
 * key arrays may be refilled between launches; their addresses and sizes are
 * fixed. */
typedef struct lp_batch lp_batch;
lp_status lp_batch_create(lp_ctx *ctx, const lp_segment_u64 *segs, uint32_t count,
                          uint64_t seed, uint64_t *d_splits, cudaStream_t stream,
                          lp_batch **out);
lp_status lp_batch_launch(lp_batch *batch, cudaStream_t stream);
/* Waits for `stream` (the stream of the batch's last launch) and returns that
 * launch's device status, as lp_ctx_wait. */
lp_status lp_batch_wait(lp_batch *batch, cudaStream_t stream);
lp_status lp_batch_destroy(lp_batch *batch);

/* Autotuner: times candidate tunings on a synthetic batch with the given
 * segment sizes (uniform keys, pivot = the middle of the key range), in a
 * temporary buffer, and stores the fastest in ctx (also returned in *best).
 * Takes a few hundred milliseconds; allocates and frees the temporary
 * buffer. */
lp_status lp_autotune_batched_u64(lp_ctx *ctx, const uint64_t *sizes, uint32_t count,
                                  cudaStream_t stream, lp_batch_tuning *best);
lp_status lp_ctx_set_batch_tuning(lp_ctx *ctx, const lp_batch_tuning *tuning);

/* ------------------------------------------------------------ quicksort
 * Sorts keys[0..n) ascending in place: the quicksort of Sec. 5 ("A Full
 * Quicksort") built on the partition.  Level-synchronous: every level
 * partitions all open subarrays (more than 4096 keys) at once through the
 * batched engine, each by [x <= p] with p the median of three keys at
 * positions drawn from `seed` and the subarray's place and level; a subarray
 * where no key exceeds p is partitioned again by [x < p] and the keys equal to
 * p are final (the paper is silent on pivots and duplicates).  Subarrays of at
 * most 4096 keys are sorted by one CTA each in shared memory (a bucket sort on
 * the subarray's key range, or a merge sort when the keys bunch).  Once a
 * level holds at most 4096 open subarrays, fewer than a quarter of the most
 * any level held, none of more than 131072 keys, each of them is sorted
 * completely by one CTA (Partial
 * Partition Steps by its warps, on-chip partitions, the shared-memory sort)
 * in one launch, instead of a level at a time.  The result
 * is the sorted array, whatever the seed; the seed only changes the work done.
 * Scratch: about 100 bytes per 4096 keys plus ~2.4 MB at most of per-segment
 * records, held by ctx.  Synchronises `stream` once per level (the host reads
 * the list sizes) and before returning.  Errors: LP_ERR_INVALID_ARG
 * (null or misaligned array), LP_ERR_OOM, LP_ERR_TIMEOUT (a bounded device
 * wait gave up), LP_ERR_CUDA. */
lp_status lp_quicksort_u64(lp_ctx *ctx, uint64_t *keys, uint64_t n, uint64_t seed,
                           cudaStream_t stream);
lp_status lp_quicksort_u32(lp_ctx *ctx, uint32_t *keys, uint64_t n, uint64_t seed,
                           cudaStream_t stream);
/* The same with the pivot of each subarray the median of pivot_samples seeded
 * keys, 3 (as above) or 15 (fewer partition passes per key: about
 * 1.05 log2(n/4096) against 1.19).  LP_ERR_INVALID_ARG for another count. */
lp_status lp_quicksort_ex_u64(lp_ctx *ctx, uint64_t *keys, uint64_t n, uint64_t seed,
                              uint32_t pivot_samples, cudaStream_t stream);
lp_status lp_quicksort_ex_u32(lp_ctx *ctx, uint32_t *keys, uint64_t n, uint64_t seed,
                              uint32_t pivot_samples, cudaStream_t stream);

/* What the last lp_quicksort_* on ctx did.  Keys "streamed" are read once and
 * written once by a kernel: the algorithmic traffic is 2 x key bytes x keys.
 * The times are device times (CUDA events) and are set only when timing is on
 * (lp_ctx_set_timing). */
typedef struct {
  uint32_t levels;          /* partition levels (each one batched launch or more) */
  uint32_t timed;           /* 1 if the two times below were measured */
  uint64_t partition_keys;  /* keys streamed by the batched partitions, all levels */
  uint64_t sort_keys;       /* keys sorted in shared memory */
  float partition_ms;       /* device time of the partition levels */
  float sort_ms;            /* device time of the levels' shared-memory sorts */
  uint32_t tail_items;      /* open subarrays the tail kernel sorted (0: none) */
  float tail_ms;            /* device time of the tail kernel */
  uint64_t tail_keys;       /* keys streamed by the tail kernel's partitions (its
                               shared-memory sorts are in sort_keys) */
} lp_sort_stats;
lp_status lp_ctx_sort_stats(const lp_ctx *ctx, lp_sort_stats *out);

/* Keys streamed (summed over every level of every segment, plus the segments
 * finished in shared memory) by the last lp_partition_batched_u64 on ctx, or by
 * the last launch of `batch`.  Both synchronise: the first the stream of the
 * batched call, the second `stream`, which must be the stream of that launch. */
lp_status lp_ctx_last_batch_keys(lp_ctx *ctx, uint64_t *keys_out);
lp_status lp_batch_streamed_keys(lp_batch *batch, cudaStream_t stream, uint64_t *keys_out);

/* Round structure of the last batched launch (same synchronisation as
 * above): the persistent kernel works in rounds -- plan, then one Partial
 * Partition Step for every open segment as warp tasks.  For round r <
 * rounds: plan_ms[r] and task_ms[r] from device timestamps, tasks[r] = warp
 * tasks of the round (groups of multi-group steps + one-group steps). */
#define LP_MAX_ROUNDS 12
typedef struct {
  uint32_t rounds;
  uint32_t pad;
  float plan_ms[LP_MAX_ROUNDS];
  float task_ms[LP_MAX_ROUNDS];
  uint64_t tasks[LP_MAX_ROUNDS];
} lp_batch_rounds;
lp_status lp_ctx_last_batch_rounds(lp_ctx *ctx, lp_batch_rounds *out);
lp_status lp_batch_round_stats(lp_batch *batch, cudaStream_t stream, lp_batch_rounds *out);

/* ------------------------------------------------------------ serving
 * A request engine (no counterpart in the paper): partition and sort requests
 * of mixed sizes and key widths are admitted first-in first-out while a slot
 * is free and the device-memory budget holds their keys (plus, for a sort, its
 * level lists), and are run by continuous batching.  Every engine step is one
 * batched launch per key width holding the newly admitted partitions and the
 * current quicksort level of every sort in flight, then the children split and
 * the shared-memory sorts of all those sorts; requests that arrive meanwhile
 * join the next step.  A partition finishes in the step it joins, a sort after
 * as many steps as its quicksort has levels (pivots: the median of 15 seeded
 * keys, as lp_quicksort_ex_* with 15, for fewer levels), or sooner: once its
 * open subarrays are few and small (the quicksort's tail rule), the next step
 * sorts each of them completely, one CTA per subarray.  Each result is the
 * same whatever the request was batched with (a partition's offsets X follow
 * from the engine seed and the request seed only; a sort's result is the
 * sorted array).
 *
 * Keys live in one device allocation of budget_bytes made at creation (the
 * arena); a request's keys are generated on the device from its seed (uniform
 * keys, as lp_fill_uniform_*), or copied from d_src, when it is admitted.  The
 * server owns an lp_ctx and a stream of its own; calls on one server must come
 * from one thread.  lp_server_step runs one engine step and synchronises. */
typedef struct lp_server lp_server;

typedef struct {
  uint64_t budget_bytes;  /* device memory for request keys and sort lists */
  uint32_t max_slots;     /* requests admitted at once, at most (0: 256) */
  uint32_t max_segments;  /* segment records per key width per step (0: 65536) */
  uint64_t seed;          /* seeds the offsets X of every batched launch */
  uint32_t keep_results;  /* 1: finished requests keep their keys until lp_server_release */
  uint32_t timing;        /* 1: CUDA events time every batched launch (stats.batched_ms) */
} lp_server_config;

enum { LP_REQ_PARTITION = 0, LP_REQ_SORT = 1 };
enum { LP_SERVE_CONTINUOUS = 0, LP_SERVE_ONE_AT_A_TIME = 1 };

typedef struct {
  uint32_t kind;       /* LP_REQ_PARTITION or LP_REQ_SORT */
  uint32_t key_bits;   /* 32 or 64 */
  uint64_t n;
  uint64_t pivot;      /* partition: dec(x) = [x <= pivot] */
  uint64_t seed;       /* names the request; the keys' generator seed when d_src is NULL */
  const void *d_src;   /* device keys copied in on admission (keep them unchanged until
                          the request is admitted), or NULL */
  double arrival_s;    /* server clock (lp_server_now); in lp_server_run: since the run began */
} lp_request;

typedef struct {
  uint64_t id;
  uint32_t kind, key_bits;
  uint64_t n;
  uint64_t split;      /* partition: keys <= pivot */
  double arrival_s, admit_s, done_s;  /* server clock */
  uint32_t steps;      /* engine steps the request took part in */
  uint32_t pad;
} lp_completion;

typedef struct {
  uint64_t steps, launches, completed, keys_done;
  uint64_t peak_bytes;    /* arena bytes in use, at most */
  uint64_t budget_bytes, in_use_bytes, engine_bytes;
  double busy_s;          /* host time spent in engine steps */
  double batched_ms;      /* device time of the batched launches (config.timing) */
} lp_server_stats;

/* Errors: LP_ERR_INVALID_ARG (bad config), LP_ERR_OOM (the budget or the
 * engine's ~20 MB of tables cannot be allocated), LP_ERR_CUDA. */
lp_status lp_server_create(int device, const lp_server_config *cfg, lp_server **out);
lp_status lp_server_destroy(lp_server *server);
const char *lp_server_last_error(const lp_server *server);
double lp_server_now(const lp_server *server);
/* Queues a request (host only).  LP_ERR_INVALID_ARG: bad kind or width, a
 * request larger than the budget, or a sort with more than max_segments *
 * 4097 keys. */
lp_status lp_server_submit(lp_server *server, const lp_request *req, uint64_t *id_out);
/* Admits what fits, runs one engine step, synchronises; *in_flight_out =
 * requests admitted and not finished.  After a device error the server
 * refuses further steps (LP_ERR_TIMEOUT / LP_ERR_CUDA). */
lp_status lp_server_step(lp_server *server, uint32_t *in_flight_out);
/* Moves up to cap finished requests' records to out, oldest first. */
lp_status lp_server_poll(lp_server *server, lp_completion *out, uint32_t cap, uint32_t *got);
/* keep_results: device address of a finished request's keys; fetch copies
 * the first `bytes` of them to dst (host or device memory, synchronous);
 * release frees them. */
lp_status lp_server_result(lp_server *server, uint64_t id, void **d_keys_out);
lp_status lp_server_fetch(lp_server *server, uint64_t id, void *dst, uint64_t bytes);
lp_status lp_server_release(lp_server *server, uint64_t id);
lp_status lp_server_get_stats(const lp_server *server, lp_server_stats *out);
/* Keys streamed (read once, written once) by all batched launches of the
 * engine, per key width. */
lp_status lp_server_streamed_keys(lp_server *server, uint64_t *keys_u64, uint64_t *keys_u32);
/* Open-loop driver: submits reqs[i] at arrival_s seconds after the call
 * begins (arrivals in time order), steps the engine until every request is
 * done and writes request i's record to out[i].  LP_SERVE_ONE_AT_A_TIME runs
 * the same requests one at a time in arrival order through lp_partition_* and
 * lp_quicksort_* instead (the per-request baseline). */
lp_status lp_server_run(lp_server *server, const lp_request *reqs, uint32_t count,
                        uint32_t mode, lp_completion *out);

/* ------------------------------------------------------------ diagnostics
 * Runs one kernel that waits on an mbarrier phase nothing completes and on a
 * grid barrier for two CTAs in a grid of one: both waits must give up after
 * the library's limit (about one second each) -- the mechanism behind
 * LP_ERR_TIMEOUT -- and the device stays usable.  *mbar_gave_up and
 * *grid_gave_up receive 1 when the respective wait gave up.  Takes about two
 * seconds; synchronises the device. */
lp_status lp_selftest_bounded_waits(int device, uint32_t *mbar_gave_up, uint32_t *grid_gave_up);

/* ------------------------------------------ Blocked-Prefix-Sum partition
 * The low-space partition of Sec. 3 with explicit block size: count the
 * predecessors (swapping the roles on the reversed array when they are the
 * majority), MakeSuccessorHeavy (Lemma 3.1), per-block predecessor counts and
 * their prefix in floor(n/B) explicit 8-byte counters (as the paper's
 * implementation stores them, Sec. 5), then Reorder (the reordering lemma)
 * from the innermost prefix outward.  base_keys == 0 finishes the innermost
 * prefix at the paper's size (at most 5B keys); a larger value finishes it on
 * chip once it has at most base_keys keys (capped by what the device's shared
 * memory holds).  LP_LOWSPACE in lp_partition_* is this call with B = 4096.
 * Scratch: about 8n/B bytes plus 8 bytes per CTA, held by ctx.  *split_out
 * (host) receives t; synchronises `stream`. */
lp_status lp_lowspace_partition_u64(lp_ctx *ctx, uint64_t *keys, uint64_t n, uint64_t pivot,
                                    uint64_t B, uint64_t base_keys, cudaStream_t stream,
                                    uint64_t *split_out);
lp_status lp_lowspace_partition_u32(lp_ctx *ctx, uint32_t *keys, uint64_t n, uint32_t pivot,
                                    uint64_t B, uint64_t base_keys, cudaStream_t stream,
                                    uint64_t *split_out);

/* ------------------------------------------------------------ host arrays
 * Partitions keys[0..n), an array in HOST memory, in place: the same split t
 * and postcondition as lp_partition_*.  The array travels to the device in
 * chunks of about n/32 keys (at least 2^22), each partitioned there in place
 * by the Smoothed Striding partition (Sec. 4) as soon as it arrives, while
 * the predecessors and successors of the chunks already done are copied back
 * to their final places: predecessors fill the host array from the front,
 * successors from the back, and a host position is written only after its
 * own chunk has reached the device.  Which end the next chunk comes from is
 * decided by the counts of earlier chunks, so the result depends on the input
 * and seed only.  Pinned host memory (cudaHostAlloc / cudaHostRegister) lets
 * the copies in both directions and the partitions overlap; pageable memory
 * works, serialised.  Device memory: a copy of the array (n keys), kept by
 * ctx for later calls and freed by lp_ctx_destroy, plus the usual scratch.
 * Ordered after earlier work on `stream`; returns when the host array holds
 * the result (it synchronises).  *split_out (host) receives t.
 * Errors: LP_ERR_INVALID_ARG for a null array with n > 0, a misaligned array
 * or a null split_out; LP_ERR_OOM when the device copy cannot be allocated;
 * LP_ERR_TIMEOUT / LP_ERR_CUDA as for lp_partition_*, after which the host
 * array's content is unspecified. */
lp_status lp_partition_host_u64(lp_ctx *ctx, uint64_t *keys, uint64_t n, uint64_t pivot,
                                uint64_t seed, cudaStream_t stream, uint64_t *split_out);
lp_status lp_partition_host_u32(lp_ctx *ctx, uint32_t *keys, uint64_t n, uint32_t pivot,
                                uint64_t seed, cudaStream_t stream, uint64_t *split_out);

/* ------------------------- Blocked-Prefix-Sum partition, values in key order
 * The fully in-place form of Sec. 3 (An Implicit Parallel Prefix Sum; In-Place
 * Reordering; Lemma bitstore2, which allows repeated keys): the same phases as
 * lp_lowspace_partition_*, but block i keeps the number of predecessors
 * before it in the order of its own first 4L + 2 keys (L = ceil(log2(n+1))),
 * not in a counter array.  Of its 2L + 1 adjacent pairs, the first write
 * moves the more common kind first (keeping their order): unequal pairs hold
 * one bit each in their order (first > second <=> 1); otherwise the second
 * keys of equal pairs 1..L are overwritten with the bits and are put back
 * when the block is read.  Auxiliary device memory: 8 bytes per CTA plus the
 * context's fixed words, whatever n.
 * B: block size, at least 4L + 2 (0 selects exactly 4L + 2, the paper's
 * size); n < 2^40.  base_keys as in lp_lowspace_partition_*.  Keys only.
 * Errors: LP_ERR_INVALID_ARG for a null or misaligned array with n > 0, a
 * null split_out, B below 4L + 2 or n >= 2^40.  *split_out (host) receives
 * t; synchronises `stream`. */
lp_status lp_lowspace_implicit_partition_u64(lp_ctx *ctx, uint64_t *keys, uint64_t n,
                                             uint64_t pivot, uint64_t B, uint64_t base_keys,
                                             cudaStream_t stream, uint64_t *split_out);
lp_status lp_lowspace_implicit_partition_u32(lp_ctx *ctx, uint32_t *keys, uint64_t n,
                                             uint32_t pivot, uint64_t B, uint64_t base_keys,
                                             cudaStream_t stream, uint64_t *split_out);
/* The first three phases only (count and role swap, MakeSuccessorHeavy, the
 * prefix phase): keys[0..n) is left as the reordering phase would find it,
 * every block's value encoded in its keys, in the logical order of the role
 * (reversed when the predecessors are the majority, 2(n - t) < n).  Exposes
 * the intermediate state; same arguments and errors as above. */
lp_status lp_lowspace_implicit_prefix_u64(lp_ctx *ctx, uint64_t *keys, uint64_t n,
                                          uint64_t pivot, uint64_t B, cudaStream_t stream,
                                          uint64_t *split_out);
lp_status lp_lowspace_implicit_prefix_u32(lp_ctx *ctx, uint32_t *keys, uint64_t n,
                                          uint32_t pivot, uint64_t B, cudaStream_t stream,
                                          uint64_t *split_out);

/* ------------------------------------------------- one Partial Partition Step
 * Runs exactly one Partial Partition Step (Sec. 4, "Formal Algorithm
 * Description"; Proposition 4.2) on keys[0..n) with explicit parameters:
 * lines of b keys, g groups, chunk j's offset X[j] = floor(r_j * g / 2^64)
 * where r_j is output j of SplitMix64 started at sigma, and sigma is output
 * `level` of SplitMix64 started at `seed` (strided != 0 forces X == 0).
 * Group i holds line j*g + (X[j]+i) mod g of every chunk j; lines past the end
 * are virtual.  Each group ends predecessors-first in its own slot order.
 * Results (host): *vmin / *vmax = min / max over non-empty groups of v_i, the
 * position of group i's first successor slot (one past its last slot when it
 * has none); *count = number of predecessors.  Afterwards keys[p] <= pivot
 * for p < vmin and keys[p] > pivot for p >= vmax.
 * Requires keys 16-byte aligned, n * sizeof(key) and b * sizeof(key)
 * multiples of 16, b * sizeof(key) <= 2048, g >= 1; otherwise
 * LP_ERR_MISALIGNED / LP_ERR_INVALID_ARG.  Synchronises `stream`. */
lp_status lp_smoothed_step_u64(lp_ctx *ctx, uint64_t *keys, uint64_t n, uint64_t pivot,
                               uint64_t b, uint64_t g, uint64_t seed, uint64_t level,
                               int strided, cudaStream_t stream, uint64_t *vmin,
                               uint64_t *vmax, uint64_t *count);
lp_status lp_smoothed_step_u32(lp_ctx *ctx, uint32_t *keys, uint64_t n, uint32_t pivot,
                               uint64_t b, uint64_t g, uint64_t seed, uint64_t level,
                               int strided, cudaStream_t stream, uint64_t *vmin,
                               uint64_t *vmax, uint64_t *count);

/* ------------------------------------------------- allocation-free variant
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory where they need a partition -- code
 * running inside another allocator's callback, latency-bound loops that must
 * not pay cudaMalloc's implicit device synchronisation, processes whose
 * device memory is entirely held by a framework's caching pool.  Such callers
 * cannot create an lp_ctx, which allocates its scratch.
 *
 * lp_partition_u64_noalloc partitions keys[0..n) on the current device with the
 * Recursive Smoothed Striding kernels of lp_partition_u64_async and writes the
 * split t to the device word *d_split when the stream gets there; it calls no
 * cudaMalloc, cudaFree or other allocating routine.  Variants: LP_SMOOTHED, as
 * lp_partition_u64_async except that a range still open at the last level is
 * finished by one group (one warp) instead of being handed to the low-space
 * partition, whose counters grow with n and have no room here; LP_STRIDED, the
 * Strided Algorithm's first step (X == 0) followed by the same Smoothed
 * Striding recursion on its open range -- not lp_partition_u64_async's
 * LP_STRIDED, which cleans that range with the low-space partition.  Both give
 * the same split and the same two sides (as multisets) as every other
 * partition of the array.  Its scratch (the
 * per-level descriptors, a status word, a grid barrier and one word per CTA
 * of the launch: about 2 KB on a 152-SM GPU, independent of n) lives in one
 * file-scope __device__ array of LP_NOALLOC_SCRATCH_BYTES bytes, which every
 * GPU that loads this library keeps until the process exits.  The first call on a device resolves that array's device address
 * and the launch grid (cudaGetSymbolAddress, occupancy queries); make that
 * first call before capturing the stream into a CUDA graph.  All calls on a
 * device share the one array: calls whose work overlaps on the GPU (other
 * streams, or graphs launched concurrently) race on it and must be
 * serialised by the caller.  Each call re-initialises the scratch it reads.
 * A device-side failure (a bounded wait that gave up) leaves *d_split =
 * UINT64_MAX, never a valid split; argument errors are
 * LP_ERR_INVALID_ARG, and so is a device whose launch grid would need more
 * scratch than the array holds (more than about 700 CTAs); CUDA failures are
 * LP_ERR_CUDA. */
#define LP_NOALLOC_SCRATCH_BYTES 4096
lp_status lp_partition_u64_noalloc(uint64_t *keys, uint64_t n, uint64_t pivot,
                                   lp_variant variant, uint64_t seed, cudaStream_t stream,
                                   uint64_t *d_split);

/* ------------------------------------------------------- synthetic inputs
 * Fill d_keys[0..n) with outputs 0..n-1 of SplitMix64 started at `seed`
 * (Steele, Lea, Flood 2014); the u32 form keeps the low 32 bits.  These are
 * the seeded uniform inputs of the benchmark workloads, not part of the
 * partition. */
lp_status lp_fill_uniform_u64(uint64_t *d_keys, uint64_t n, uint64_t seed,
                              cudaStream_t stream);
lp_status lp_fill_uniform_u32(uint32_t *d_keys, uint64_t n, uint64_t seed,
                              cudaStream_t stream);
/* d_vals[i] = i. */
lp_status lp_fill_iota_u64(uint64_t *d_vals, uint64_t n, cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* LIBPARTITION_H */
