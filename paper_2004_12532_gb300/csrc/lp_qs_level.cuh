// lp_qs_level.cuh -- one level of the quicksort on the partition (Sec. 5, "A
// Full Quicksort") item by item: the segment record of an open subarray (its
// pivot) and its children after the partition, for the per-level kernels of
// lp_qs.cu.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "lp_qs.cuh"
#include "lp_qs_pivot.cuh"

namespace lp {

// The caller's fields of the segment record of item q at `level` of a sort
// seeded with `seed`: a normal item's pivot is the median of `samples` (3 or
// 15) seeded keys, an equal-key item's the equal key minus one; the salt (the
// seed of the segment's offsets X) is named by the subarray and the level,
// not by its place in the list.
template <typename T>
__device__ __forceinline__ SegDesc qs_item_record(T* keys, const QsItem& q, uint64_t seed,
                                                  uint32_t level, uint32_t samples) {
  const uint64_t h = qs_item_hash(seed, level, q.lo, q.n);
  SegDesc d = {};
  d.keys = keys + q.lo;
  d.n = q.n;
  if (q.eq) {
    d.pivot = q.pivot - 1;  // q.pivot > 0: a zero pivot never makes an equal-key item
  } else {
    d.pivot = (uint64_t)(samples == kQsSamplesMax ? qs_median<kQsSamplesMax>(keys, q.lo, q.n, h)
                                                  : qs_median<3>(keys, q.lo, q.n, h));
  }
  d.salt = sm_stream(h, kQsSamplesMax + 1);
  return d;
}

// A child [lo, lo + n) of an item of J's level: to the small list (sorted in
// shared memory) or to the next level's list.
__device__ __forceinline__ void qs_push(const QsJob& J, uint64_t lo, uint64_t n) {
  if (n <= 1) return;  // a single key is in place
  if (n <= (J.local_cut ? (uint64_t)J.local_cut : kQsCut)) {
    J.small[atomicAdd(&J.lc->small, 1u)] = QsSmall{lo, (uint32_t)n, J.level + 1};
    atomicAdd(J.sort_keys, (unsigned long long)n);
  } else {
    J.next[atomicAdd(&J.lc->next, 1u)] = QsItem{lo, n, 0, 0};
    atomicMax(&J.lc->max_next, n < 0xffffffffull ? (uint32_t)n : 0xffffffffu);
  }
}

// The children of item q, partitioned with split t by `pivot`.
__device__ __forceinline__ void qs_item_children(const QsJob& J, const QsItem& q, uint64_t t,
                                                 uint64_t pivot) {
  if (q.eq) {  // [lo, lo + t) < p; the rest equals p
    qs_push(J, q.lo, t);
    return;
  }
  if (t == q.n) {  // no successor: split off the keys equal to the pivot next level
    if (pivot != 0) {
      J.next[atomicAdd(&J.lc->next, 1u)] = QsItem{q.lo, q.n, pivot, 1};
      atomicMax(&J.lc->max_next, q.n < 0xffffffffull ? (uint32_t)q.n : 0xffffffffu);
    }
    return;
  }
  qs_push(J, q.lo, t);
  qs_push(J, q.lo + t, q.n - t);
}

}  // namespace lp
