// lp_batched.h -- internal interface of the batched partition engine
// (lp_batched.cu): per-segment device records, scratch layout, tuning knobs.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

#include "lp_launch.h"

namespace lp {

// One segment of a batch, in device memory.  The first four fields are the
// caller's; the rest is the engine's state.
struct SegDesc {
  void* keys;
  uint64_t n;
  uint64_t pivot;
  uint64_t salt;                    // names the segment: its offsets X depend on it
  uint64_t seed;                    // per-segment seed of the offsets X (batch seed, salt)
  uint64_t h, be;                   // 16-byte aligned body [h, be)
  uint64_t lo, hi;                  // open range of the current level
  uint64_t b, g;                    // step parameters of the current level
  unsigned long long vmin, vmax;    // this level's v_min / v_max (atomics)
  unsigned long long count;         // this level's predecessor count (atomics)
  unsigned long long body_count;    // predecessors of the body (from level 0)
  unsigned long long t;             // the split, once done
  uint32_t level, state;
  uint32_t staged;                  // multi-CTA finish: slices staged on chip so far
  uint32_t spare;
};

// Open ranges of at most this many bytes get a one-group step: one warp
// partitions the whole range.
constexpr uint32_t kWarpCapBytes = 128u * 1024u;
// CTAs of a batched launch, at most (plan space per CTA)
constexpr uint32_t kBatchMaxGrid = 1024;
// task kinds a plan counts per CTA
constexpr uint32_t kPlanKinds = 6;
// slices of multi-CTA finishes per window (their counts' space); a grid
// barrier separates windows
constexpr uint32_t kMcWindow = 16384;
static_assert(kMcWindow >= 4 * kBatchMaxGrid, "a window holds any finish");
// rounds recorded in BatchScratch::tround
constexpr uint32_t kBatchRoundSlots = 12;

struct BatchArgs {
  uint64_t* splits;       // one split per segment (device)
  uint32_t max_rounds;
  uint64_t group_workers; // at most this many groups per segment step
  uint32_t line_bytes;    // line size of the steps
  uint32_t min_chunks;    // lines per group, at least
  uint64_t warp_cap;      // one-group steps for open ranges of at most this many keys
  uint32_t min_chunks_residual;  // lines per group, at least, after the first step
  uint32_t mc_slices;     // multi-CTA finishes span at most this many slices (<= grid)
  uint32_t mc_window;     // slices per window of their counts (>= mc_slices)
};

struct BatchScratch {
  unsigned long long* mprefix;  // multi-group segments: prefix of their group counts
  uint32_t* mseg;               // multi-group segments: ids
  uint32_t* singles;            // one-group segments: ids
  uint32_t* ctalist;            // CTA-task segments: ids
  uint32_t* mcprefix;           // multi-CTA finishes: prefix of their CTA slices
  uint32_t* mcseg;              // multi-CTA finishes: ids
  uint32_t* mccount;            // per slice of a window: its predecessor count
  uint32_t* cta_tot;            // per CTA: singles, groups, multi-group segments, CTA tasks,
                                // multi-CTA slices, multi-CTA segments
  unsigned long long* totals;   // [2]: keys streamed
  unsigned long long* tround;   // per round: plan start, tasks start, tasks end (ns), tasks
  uint32_t* counters;           // task fetch counters: warp tasks, CTA tasks, slices (2)
  uint32_t* bar;                // grid barrier
  uint32_t* status;
};

// Knobs the autotuner sets (0: default).
struct BatchTuning {
  uint32_t ctas;           // CTAs of the persistent launch
  uint64_t group_workers;  // groups per segment step, at most
  uint32_t line_bytes;     // 128..1024
  uint32_t min_chunks;     // lines per group, at least
  uint32_t min_chunks_residual;  // ... in steps after the first
  uint32_t mc_slices;      // multi-CTA finishes span at most this many slices; below the
                           // grid it also cuts their windows to 4x that (tests)
};

size_t batch_scratch_bytes(uint32_t count);
BatchScratch carve_batch_scratch(void* base, uint32_t count, uint32_t* bar, uint32_t* status);

// Sets the batched kernel's shared-memory attribute (once per device, before
// any stream capture) and returns its cooperative grid: SMs x resident CTAs.
template <typename T>
cudaError_t batched_prepare(int device, uint32_t* grid);

// One persistent launch over the segments, after a set-up launch that gives
// every record its engine state and resets the grid barrier and the tallies
// (lp_batch_init.cuh); with records_ready the caller has done that on the
// device already (for `seed`) and only the persistent launch runs.  The
// status word is not reset (a caller resets it once per call, so a failure of
// any launch of the call stays visible).
template <typename T>
cudaError_t launch_batched(SegDesc* d_segs, uint32_t count, uint64_t seed, uint64_t* d_splits,
                           const BatchScratch& B, const BatchTuning& tune, LaunchCfg& cfg,
                           bool records_ready = false);

// Quicksort on the batched partition (lp_quicksort.cu).  `staging`:
// quicksort_staging_bytes(n) of pinned host memory for the per-level job
// records and read-backs; synchronises `cfg.stream` once per level.  `ev`
// (three events, or null) times the partition levels and the shared-memory
// sorts.
struct SortStats {
  uint32_t levels;          // level-synchronous levels
  uint64_t partition_keys;  // keys streamed by their batched partitions
  uint64_t sort_keys;       // keys sorted in shared memory (levels and tail)
  float partition_ms, sort_ms;
  uint32_t tail_items;      // subarrays the tail kernel finished (0: no tail)
  uint64_t tail_keys;       // keys streamed by the tail kernel's partitions
  float tail_ms;            // its device time
};

size_t quicksort_scratch_bytes(uint64_t n);
size_t quicksort_staging_bytes(uint64_t n);

// `samples`: pivot = the median of 3 or 15 seeded keys per subarray.
template <typename T>
cudaError_t launch_quicksort(T* keys, uint64_t n, uint64_t seed, uint32_t samples, void* scratch,
                             void* staging, const BatchTuning& tune, uint32_t* bar,
                             uint32_t* status, LaunchCfg& cfg, const cudaEvent_t* ev,
                             SortStats* stats);

}  // namespace lp
