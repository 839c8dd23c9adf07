// lp_qs.cuh -- device side of the quicksort on the partition (Sec. 5, "A
// Full Quicksort"), shared by the one-array quicksort (lp_quicksort.cu) and
// the serving engine (lp_server.cu), which runs the levels of many sorts in
// the same batched launches.
//
// A sort job owns an item list per level.  An item is an open subarray
// [lo, lo + n) with n > kQsCut:
//   normal item: partitioned by [x <= p], p the median of three keys at seeded
//                positions; children of at most kQsCut keys go to the job's
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
constexpr uint32_t kQsSortThreads = 512;

struct QsItem {
  uint64_t lo, n, pivot;  // pivot: of an equal-key item only
  uint64_t eq;            // 1: equal-key item
};
struct QsSmall {
  uint64_t lo, n;
};
// per-job list sizes of the current level (reset every level), in device memory
struct QsLevelCounts {
  uint32_t next, small;
};

// One slice of one job's list in one launch.
struct QsJob {
  void* keys;                      // the job's array
  const QsItem* items;             // this slice of the level's list
  QsItem* next;                    // the next level's list (whole job)
  QsSmall* small;                  // the level's small list (whole job)
  QsLevelCounts* lc;               // the job's level counts
  unsigned long long* sort_keys;   // keys the job sorted in shared memory, accumulated
  uint64_t seed;                   // the job's seed (pivots and offsets X)
  uint32_t level;                  // the job's current level
  uint32_t count;                  // items in this slice
  uint32_t seg_base;               // index of the slice's first segment record
  uint32_t pad;
};

template <typename T>
__device__ __forceinline__ T qs_ld(const T* p) {
  if constexpr (sizeof(T) == 8) return (T)__ldcg(reinterpret_cast<const unsigned long long*>(p));
  else return (T)__ldcg(reinterpret_cast<const unsigned int*>(p));
}

// Segment records of every job slice: blockIdx.y = job, x = item.
template <typename T>
__global__ void qs_build_kernel(const QsJob* jobs, SegDesc* segs) {
  const QsJob& J = jobs[blockIdx.y];
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= J.count) return;
  const QsItem q = J.items[i];
  T* keys = static_cast<T*>(J.keys);
  const uint64_t h = sm_stream(J.seed + J.level, q.lo ^ (q.n << 32));
  SegDesc d = {};
  d.keys = keys + q.lo;
  d.n = q.n;
  if (q.eq) {
    d.pivot = q.pivot - 1;  // q.pivot > 0: a zero pivot never makes an equal-key item
  } else {
    const T a = qs_ld(&keys[q.lo + range_of(sm_stream(h, 0), q.n)]);
    const T b = qs_ld(&keys[q.lo + range_of(sm_stream(h, 1), q.n)]);
    const T c = qs_ld(&keys[q.lo + range_of(sm_stream(h, 2), q.n)]);
    const T mx = a > b ? a : b, mn = a > b ? b : a;
    d.pivot = (uint64_t)(c > mx ? mx : (c < mn ? mn : c));
  }
  d.salt = sm_stream(h, 3);  // the subarray and level name it, not its place in the list
  segs[J.seg_base + i] = d;
}

static __device__ __forceinline__ void qs_push(const QsJob& J, uint64_t lo, uint64_t n) {
  if (n <= 1) return;  // a single key is in place
  if (n <= kQsCut) {
    J.small[atomicAdd(&J.lc->small, 1u)] = QsSmall{lo, n};
    atomicAdd(J.sort_keys, (unsigned long long)n);
  } else {
    J.next[atomicAdd(&J.lc->next, 1u)] = QsItem{lo, n, 0, 0};
  }
}

// Children of every partitioned item (after the batched launch); the keys the
// launch streamed are added to *traffic_acc.
static __global__ void qs_split_kernel(const QsJob* jobs, const SegDesc* segs, const uint64_t* splits,
                                const unsigned long long* traffic,
                                unsigned long long* traffic_acc) {
  const QsJob& J = jobs[blockIdx.y];
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *traffic_acc += *traffic;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= J.count) return;
  const QsItem q = J.items[i];
  const uint64_t t = splits[J.seg_base + i];
  if (q.eq) {  // [lo, lo + t) < p; the rest equals p
    qs_push(J, q.lo, t);
    return;
  }
  if (t == q.n) {  // no successor: split off the keys equal to the pivot next level
    const uint64_t p = segs[J.seg_base + i].pivot;
    if (p != 0) J.next[atomicAdd(&J.lc->next, 1u)] = QsItem{q.lo, q.n, p, 1};
    return;
  }
  qs_push(J, q.lo, t);
  qs_push(J, q.lo + t, q.n - t);
}

// Every job's small list, one subarray per CTA at a time: bitonic sorting
// network in shared memory over the next power of two, padded with the
// largest key; blockIdx.y = job.  The list size is read on the device.
template <typename T>
__global__ void __launch_bounds__(kQsSortThreads) qs_small_sort_kernel(const QsJob* jobs) {
  __shared__ T buf[kQsCut];
  const QsJob& J = jobs[blockIdx.y];
  const uint32_t tid = threadIdx.x;
  const uint32_t cnt = *reinterpret_cast<volatile uint32_t*>(&J.lc->small);
  T* keys = static_cast<T*>(J.keys);
  for (uint32_t s = blockIdx.x; s < cnt; s += gridDim.x) {
    const QsSmall q = J.small[s];
    const uint32_t n = (uint32_t)q.n;
    uint32_t P = 2;
    while (P < n) P <<= 1;
    for (uint32_t i = tid; i < P; i += kQsSortThreads)
      buf[i] = i < n ? qs_ld(&keys[q.lo + i]) : (T)~(T)0;
    __syncthreads();
    for (uint32_t k = 2; k <= P; k <<= 1) {
      for (uint32_t j = k >> 1; j > 0; j >>= 1) {
        // pair p: i = the p-th index with bit j clear, partner i + j
        for (uint32_t p = tid; p < (P >> 1); p += kQsSortThreads) {
          const uint32_t i = ((p & ~(j - 1)) << 1) | (p & (j - 1));
          const uint32_t l = i + j;
          const T x = buf[i], y = buf[l];
          const bool up = (i & k) == 0;
          if ((x > y) == up) { buf[i] = y; buf[l] = x; }
        }
        __syncthreads();
      }
    }
    for (uint32_t i = tid; i < n; i += kQsSortThreads) keys[q.lo + i] = buf[i];
    __syncthreads();
  }
}

}  // namespace lp
