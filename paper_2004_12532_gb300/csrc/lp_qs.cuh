// lp_qs.cuh -- the quicksort on the partition (Sec. 5, "A Full Quicksort"):
// records and kernel launchers (kernels in lp_qs.cu) shared by the one-array
// quicksort (lp_quicksort.cu) and the serving engine (lp_server.cu), which
// runs the levels of many sorts in the same batched launches.
//
// A sort job owns an item list per level.  An item is an open subarray
// [lo, lo + n) with n > kQsCut:
//   normal item: partitioned by [x <= p], p the median of 3 (or 15) keys at
//                seeded positions; children of at most kQsCut keys go to the job's
//                small list, larger ones to the next level's list; if no key
//                exceeds p (t = n) and p > 0, the subarray comes back at the
//                next level as an equal-key item;
//   equal-key item: partitioned by [x < p] (pivot p - 1); [lo, lo + t') is a
//                normal child, the keys equal to p are in final place.
// The subarrays of one level are disjoint and hold more than kQsCut keys, so
// a list never holds more than n / (kQsCut + 1) items.  Small subarrays are
// sorted by one CTA each in shared memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "lp_batched.h"
#include "lp_plan.h"

namespace lp {

constexpr uint64_t kQsCut = 4096;  // subarrays this small are sorted in shared memory
constexpr uint32_t kQsSortThreads = 256;
constexpr uint32_t kQsSamplesMax = 15;  // pivot samples per subarray, at most

struct QsItem {
  uint64_t lo, n, pivot;  // pivot: of an equal-key item only
  uint64_t eq;            // 1: equal-key item
};
struct QsSmall {
  uint64_t lo;
  uint32_t n;      // at most kQsCut (or the job's local_cut)
  uint32_t level;  // the subarray's level (names its pivot when it is partitioned further)
};
// per-job list sizes of the current level (reset every level), in device memory
struct QsLevelCounts {
  uint32_t next, small;
  uint32_t max_next;  // keys of the largest item of the next list (saturated at 2^32 - 1)
  uint32_t merge;     // small subarrays the bucket sort left to the merge sort
};

// One slice of one job's list in one launch.
struct QsJob {
  void* keys;                      // the job's array
  const QsItem* items;             // this slice of the level's list
  QsItem* next;                    // the next level's list (whole job)
  QsSmall* small;                  // the level's small list (whole job)
  uint32_t* merge;                 // indices into it: the merge sort's subarrays (room
                                   // for as many entries as the small list)
  QsLevelCounts* lc;               // the job's level counts
  unsigned long long* sort_keys;   // keys the job sorted in shared memory, accumulated
  uint64_t seed;                   // the job's seed (pivots and offsets X)
  uint32_t level;                  // the job's current level
  uint32_t count;                  // items in this slice
  uint32_t seg_base;               // index of the slice's first segment record
  uint32_t samples;                // pivot: median of this many seeded keys (3 or 15; 0: 3)
  uint32_t local_cut;              // children of at most this many keys go to the small
                                   // list (0: kQsCut, the shared-memory sort's size)
};

// Segment records of every job in `jobs` (grid.y = jobs, x covers the
// largest item count): median-of-3 (or -15) pivots, equal-key pivots minus one.
template <typename T>
cudaError_t launch_qs_build(const QsJob* jobs, uint32_t njobs, uint32_t max_count, SegDesc* segs,
                            cudaStream_t st);

// One slice's level set-up in one launch (the one-array quicksort): writes J
// to d_job, where the level's split and sort kernels read it, resets J.lc when
// reset_counts (the level's first slice), and builds the slice's segment
// records as launch_qs_build does, with the batched engine's set-up for
// `batch_seed` (launch_batched then runs with records_ready).
template <typename T>
cudaError_t launch_qs_level_start(const QsJob& J, QsJob* d_job, SegDesc* segs,
                                  uint64_t batch_seed, const BatchScratch& B, bool reset_counts,
                                  cudaStream_t st);

// Children of every partitioned item after the batched launch; adds the keys
// that launch streamed (*traffic) to *traffic_acc.
cudaError_t launch_qs_split(const QsJob* jobs, uint32_t njobs, uint32_t max_count,
                            const SegDesc* segs, const uint64_t* splits,
                            const unsigned long long* traffic, unsigned long long* traffic_acc,
                            cudaStream_t st);

// Sorts every job's small list in shared memory; `ctas` CTAs per job.  The
// bucket sort runs here (4 CTAs per SM); a subarray whose keys bunch goes to
// the job's merge list instead, counted in lc->merge, and stays unsorted
// until launch_qs_merge_sort -- which the caller runs, when a read-back shows
// a nonzero count, before the lists are reused.
template <typename T>
cudaError_t launch_qs_small_sort(const QsJob* jobs, uint32_t njobs, uint32_t ctas,
                                 cudaStream_t st);
// The merge sort of every job's merge list.
template <typename T>
cudaError_t launch_qs_merge_sort(const QsJob* jobs, uint32_t njobs, uint32_t ctas,
                                 cudaStream_t st);

// Sets the shared-memory attribute of the sort kernels (once per device).
cudaError_t qs_prepare();

// The tail: once a level holds at most kQsTailItems open subarrays, fewer than
// 1/kQsTailDrop of the most any level of the sort held, none of more than
// kQsTailMaxKeys keys, each of them is sorted by one CTA in one launch
// (launch_qs_local) instead of a level at a time -- the last levels hold few
// keys and would each cost a level's fixed overhead (or, in the serving
// engine, an engine step).
constexpr uint64_t kQsTailItems = 4096;
constexpr uint64_t kQsTailDrop = 4;
constexpr uint64_t kQsTailMaxKeys = 131072;
inline bool qs_is_tail(uint64_t open, uint64_t peak_open, uint64_t max_item) {
  return open > 0 && open <= kQsTailItems && open * kQsTailDrop < peak_open &&
         max_item <= kQsTailMaxKeys;
}

// The tail of a sort (lp_qs_local.cu): every item list[0..count) of level
// `level` (open subarrays, normal or equal-key) is sorted completely by one
// CTA, depth first -- Partial Partition Steps by its warps, on-chip
// partitions, then the shared-memory sort of pieces of at most kQsCut keys --
// with no grid-wide barrier.  Pivots as in the levels (qs_item_hash).
// acc[0] += keys streamed by its partitions, acc[1] += keys it sorted in
// shared memory, acc[3] / acc[4] += the CTAs' device time (ns, summed over
// CTAs) in sorts / in partitions; acc[2] is its fetch counter.  `grid`: CTAs
// (at most qs_local_grid).
template <typename T>
cudaError_t launch_qs_local(T* keys, const QsItem* list, uint32_t count, uint32_t level,
                            uint64_t seed, uint32_t samples, unsigned long long* acc,
                            uint32_t* status, uint32_t grid, cudaStream_t st);
template <typename T>
cudaError_t qs_local_grid(int device, uint32_t* grid);

}  // namespace lp
