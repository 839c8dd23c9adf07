// lp_qs_pivot.cuh -- pivots of the quicksort on the partition (Sec. 5, "A
// Full Quicksort"; the paper is silent on pivots): the median of NS keys at
// positions drawn from a hash of the job's seed, the subarray's place and its
// level.  Shared by the level-synchronous levels (lp_qs.cu) and the on-chip
// finishing kernel (lp_qs_local.cu), so a subarray gets the same pivot in
// either.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "lp_plan.h"

namespace lp {

// The hash naming subarray [lo, lo + n) at `level` of a sort seeded with `seed`.
__device__ __forceinline__ uint64_t qs_item_hash(uint64_t seed, uint32_t level, uint64_t lo,
                                                 uint64_t n) {
  return sm_stream(seed + level, lo ^ (n << 32));
}

template <typename T>
__device__ __forceinline__ T qs_ld(const T* p) {
  if constexpr (sizeof(T) == 8) return (T)__ldcg(reinterpret_cast<const unsigned long long*>(p));
  else return (T)__ldcg(reinterpret_cast<const unsigned int*>(p));
}

// The median of NS keys at seeded positions of keys[lo, lo + n): all loads
// first, then an insertion sort in registers (fully unrolled).
template <uint32_t NS, typename T>
__device__ __forceinline__ T qs_median(const T* keys, uint64_t lo, uint64_t n, uint64_t h) {
  T v[NS];
#pragma unroll
  for (uint32_t j = 0; j < NS; j++) v[j] = qs_ld(&keys[lo + range_of(sm_stream(h, j), n)]);
#pragma unroll
  for (uint32_t j = 1; j < NS; j++) {
#pragma unroll
    for (uint32_t r = j; r > 0; r--) {
      const T a = v[r - 1] < v[r] ? v[r - 1] : v[r], b = v[r - 1] < v[r] ? v[r] : v[r - 1];
      v[r - 1] = a;
      v[r] = b;
    }
  }
  return v[NS / 2];
}

}  // namespace lp
