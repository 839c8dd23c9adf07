// lp_qs_sort.cuh -- the shared-memory sort of one small subarray by one CTA
// of kQsSortThreads threads (quicksort on the partition, Sec. 5): used by the
// quicksort's sort kernel.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "lp_qs.cuh"

namespace lp {

// One CTA sorts one subarray of n <= kQsCut keys.  Thread t owns the 16 keys
// [16t, 16t + 16) of the n rounded up to 16 (the last block padded with the
// largest key): it sorts them with Batcher's odd-even merge network (63
// comparators), then merge passes double the sorted runs until one run covers
// the subarray; in each pass thread t finds where output position 16t of its
// pair of runs splits the two inputs (a binary search along the merge-path
// diagonal) and merges its 16 outputs into registers; after a barrier they
// overwrite the pass's input.  Runs live in one shared-memory buffer (35 KB
// for uint64: four CTAs per SM hide the latency of the dependent loads),
// padded by one word every 128 bytes so that the threads' 16-key blocks fall
// in distinct banks.
constexpr uint32_t kE = 16;
static_assert(kQsSortThreads * kE == kQsCut, "one CTA holds a whole small subarray");

template <typename T>
struct SortSmem {
  static constexpr uint32_t kShift = sizeof(T) == 8 ? 4 : 5;  // words per 128 bytes
  static constexpr uint32_t kWords = kQsCut + (kQsCut >> kShift);
  static constexpr size_t kBytes = kWords * sizeof(T);
  __device__ static __forceinline__ uint32_t pad(uint32_t i) { return i + (i >> kShift); }
};

template <typename T>
__device__ __forceinline__ void cswap(T& a, T& b) {
  const bool s = b < a;
  const T x = s ? b : a, y = s ? a : b;
  a = x;
  b = y;
}

// Batcher's odd-even merge sort of 16 keys (comparators in network order)
template <typename T>
__device__ __forceinline__ void sort16(T (&v)[kE]) {
  constexpr uint8_t net[63][2] = {
      {0, 1},   {2, 3},   {0, 2},   {1, 3},   {1, 2},   {4, 5},   {6, 7},   {4, 6},
      {5, 7},   {5, 6},   {0, 4},   {2, 6},   {2, 4},   {1, 5},   {3, 7},   {3, 5},
      {1, 2},   {3, 4},   {5, 6},   {8, 9},   {10, 11}, {8, 10},  {9, 11},  {9, 10},
      {12, 13}, {14, 15}, {12, 14}, {13, 15}, {13, 14}, {8, 12},  {10, 14}, {10, 12},
      {9, 13},  {11, 15}, {11, 13}, {9, 10},  {11, 12}, {13, 14}, {0, 8},   {4, 12},
      {4, 8},   {2, 10},  {6, 14},  {6, 10},  {2, 4},   {6, 8},   {10, 12}, {1, 9},
      {5, 13},  {5, 9},   {3, 11},  {7, 15},  {7, 11},  {3, 5},   {7, 9},   {11, 13},
      {1, 2},   {3, 4},   {5, 6},   {7, 8},   {9, 10},  {11, 12}, {13, 14}};
#pragma unroll
  for (int c = 0; c < 63; c++) cswap(v[net[c][0]], v[net[c][1]]);
}


// Sorts keys[0..n), n <= kQsCut, ascending, with all kQsSortThreads threads of
// the CTA (blockDim.x == kQsSortThreads); `smem` holds SortSmem<T>::kBytes.
// Ends with a CTA barrier (the buffer may be reused at once).
template <typename T>
__device__ __forceinline__ void cta_sort_small(T* __restrict__ keys, uint32_t n, unsigned char* smem) {
  using S = SortSmem<T>;
  T* const buf = reinterpret_cast<T*>(smem);
  const uint32_t tid = threadIdx.x;
  const T big = (T)~(T)0;
  const uint32_t n16 = (n + kE - 1) / kE * kE;
  const uint32_t d0 = tid * kE;  // this thread's first output position
  const bool on = d0 < n16;
  {  // coalesced load through L2, every load issued before the first store
    T x[kE];
#pragma unroll
    for (uint32_t m = 0; m < kE; m++) {
      const uint32_t i = tid + m * kQsSortThreads;
      if constexpr (sizeof(T) == 8)
        x[m] = i < n ? (T)__ldcg(reinterpret_cast<const unsigned long long*>(keys + i)) : big;
      else
        x[m] = i < n ? (T)__ldcg(reinterpret_cast<const unsigned int*>(keys + i)) : big;
    }
#pragma unroll
    for (uint32_t m = 0; m < kE; m++) {
      const uint32_t i = tid + m * kQsSortThreads;
      if (i < n16) buf[S::pad(i)] = x[m];
    }
  }
  __syncthreads();
  T v[kE];
  if (on) {
#pragma unroll
    for (uint32_t r = 0; r < kE; r++) v[r] = buf[S::pad(d0 + r)];
    sort16(v);
#pragma unroll
    for (uint32_t r = 0; r < kE; r++) buf[S::pad(d0 + r)] = v[r];
  }
  __syncthreads();
  for (uint32_t L = kE; L < n16; L <<= 1) {
    const T* src = buf;
    if (on) {
      // runs A = [base, base + LA), B = [base + LA, base + LA + LB), clipped to n16
      const uint32_t base = d0 & ~(2 * L - 1), d = d0 - base;
      const uint32_t LA = min(L, n16 - base), LB = min(L, n16 - base - LA);
      const uint32_t ab = base, bb = base + LA;
      uint32_t lo = d > LB ? d - LB : 0, hi = d < LA ? d : LA;
      while (lo < hi) {  // the merge-path split of diagonal d
        const uint32_t mid = (lo + hi) >> 1;
        if (src[S::pad(ab + mid)] <= src[S::pad(bb + d - 1 - mid)]) lo = mid + 1;
        else hi = mid;
      }
      uint32_t i = lo, j = d - lo;
      T a = i < LA ? src[S::pad(ab + i)] : big;
      T b = j < LB ? src[S::pad(bb + j)] : big;
#pragma unroll
      for (uint32_t r = 0; r < kE; r++) {
        const bool ta = j >= LB || (i < LA && a <= b);
        v[r] = ta ? a : b;
        i += ta ? 1u : 0u;
        j += ta ? 0u : 1u;
        const uint32_t ni = ta ? i : j;
        if (ni < (ta ? LA : LB)) {
          const T nx = src[S::pad((ta ? ab : bb) + ni)];
          if (ta) a = nx; else b = nx;
        }
      }
    }
    __syncthreads();  // every thread has read the pass's input
    if (on) {
#pragma unroll
      for (uint32_t r = 0; r < kE; r++) buf[S::pad(d0 + r)] = v[r];
    }
    __syncthreads();
  }
#pragma unroll
  for (uint32_t m = 0; m < kE; m++) {
    const uint32_t i = tid + m * kQsSortThreads;
    if (i < n) keys[i] = buf[S::pad(i)];
  }
  __syncthreads();
}

}  // namespace lp
