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
// comparators).  Each warp then merges its 32 runs of 16 into one run of 512
// in registers: per doubling, a bitonic "flip" stage (position p of the lower
// run against position S - 1 - p of the upper one) and half-cleaners, across
// lanes by shuffles and inside a lane by compare-exchanges -- independent
// work, no shared memory and no CTA barrier.  Merge passes then double the
// runs from 512 until one run covers the subarray; in each pass thread t finds
// where output position 16t of its pair of runs splits the two inputs (a
// binary search along the merge-path diagonal) and merges its 16 outputs into
// registers; after a barrier they overwrite the pass's input.  Runs live in
// one shared-memory buffer (35 KB for uint64), padded by one word every 128
// bytes so that the threads' 16-key blocks fall in distinct banks.
constexpr uint32_t kE = 16;
static_assert(kQsSortThreads * kE == kQsCut, "one CTA holds a whole small subarray");

template <typename T>
struct SortSmem {
  // the merge sort: one padded run buffer
  static constexpr uint32_t kShift = sizeof(T) == 8 ? 4 : 5;  // words per 128 bytes
  static constexpr uint32_t kWords = kQsCut + (kQsCut >> kShift);
  static constexpr size_t kMergeBytes = kWords * sizeof(T);
  // the bucket sort (overlays the same memory): the keys in bucket order, the
  // buckets' starts and fill positions, reduction words
  static constexpr uint32_t kBucketsMax = kQsCut / 2;
  static constexpr size_t kStartOff = (size_t)kQsCut * sizeof(T);
  static constexpr size_t kFillOff = kStartOff + ((kBucketsMax + 1) * 4 + 15) / 16 * 16;
  static constexpr size_t kRedOff = kFillOff + (size_t)kBucketsMax * 4;
  static constexpr size_t kBucketBytes = kRedOff + 256;
  static constexpr size_t kBytes = kMergeBytes > kBucketBytes ? kMergeBytes : kBucketBytes;
  __device__ static __forceinline__ uint32_t pad(uint32_t i) { return i + (i >> kShift); }
};
// A bucket holding more keys than this sends the subarray to the merge sort.
constexpr uint32_t kBucketSortMax = 32;

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


// x becomes min(x, y) when keep_min, else max(x, y).
template <typename T>
__device__ __forceinline__ void keep_one(T& x, T y, bool keep_min) {
  const bool y_less = y < x;
  x = (y_less == keep_min) ? y : x;
}

template <typename T>
__device__ __forceinline__ T shfl_xor_key(T x, uint32_t m) {
  if constexpr (sizeof(T) == 8)
    return (T)__shfl_xor_sync(0xffffffffu, (unsigned long long)x, (int)m);
  else
    return (T)__shfl_xor_sync(0xffffffffu, (unsigned int)x, (int)m);
}

// The 32 lanes of a warp hold positions [16 lane, 16 lane + 16) of 512 keys,
// each lane's 16 sorted ascending; afterwards all 512 are sorted ascending
// across the lanes.  Bitonic merging of runs S = 32 .. 512 keys (lanes = S /
// 16 lanes per run): the flip pairs position p of the lower half with S - 1 - p
// of the upper half (lane l ^ (lanes - 1), register 15 - r), the smaller
// staying below; half-cleaners at distance d pair p with p + d, across lanes
// for d >= 16 (lane distance d / 16) and inside a lane below.
template <typename T>
__device__ __forceinline__ void warp_merge_to_512(T (&v)[kE], uint32_t lane) {
#pragma unroll
  for (uint32_t lanes = 2; lanes <= 32; lanes <<= 1) {
    const bool lower = (lane & (lanes >> 1)) == 0;
#pragma unroll
    for (uint32_t r = 0; r < kE / 2; r++) {
      const T a = shfl_xor_key(v[kE - 1 - r], lanes - 1);
      const T b = shfl_xor_key(v[r], lanes - 1);
      keep_one(v[r], a, lower);
      keep_one(v[kE - 1 - r], b, lower);
    }
#pragma unroll
    for (uint32_t m = lanes >> 2; m >= 1; m >>= 1) {
      const bool lo = (lane & m) == 0;
#pragma unroll
      for (uint32_t r = 0; r < kE; r++) keep_one(v[r], shfl_xor_key(v[r], m), lo);
    }
#pragma unroll
    for (uint32_t d = kE / 2; d >= 1; d >>= 1) {
#pragma unroll
      for (uint32_t r = 0; r < kE; r++)
        if ((r & d) == 0) cswap(v[r], v[r + d]);
    }
  }
}

// CTA-wide exclusive scan of one value per thread (all kQsSortThreads threads
// call it); *total receives the sum.  `ws` holds kQsSortThreads / 32 words.
__device__ __forceinline__ uint32_t cta_scan_u32(uint32_t v, uint32_t* ws, uint32_t* total) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (uint32_t o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  __syncthreads();
  if (lane == 31) ws[warp] = incl;
  __syncthreads();
  uint32_t before = 0, all = 0;
  for (uint32_t w = 0; w < kQsSortThreads / 32; w++) {
    const uint32_t y = ws[w];
    before += w < warp ? y : 0u;
    all += y;
  }
  *total = all;
  return before + incl - v;
}

// The sort of keys[0..n), n <= kQsCut, ascending, by all kQsSortThreads
// threads of the CTA (blockDim.x == kQsSortThreads), `smem` holding
// SortSmem<T>::kBytes: a load into registers, then the bucket sort, and the
// merge sort for the subarrays the bucket sort turns down.  Each part ends
// with a CTA barrier (the buffer may be reused at once); cta_sort_small runs
// all three, and the quicksort's levels run the merge sort in a kernel of its
// own, so that the bucket sort's kernel needs fewer registers.
//
// The bucket sort: with [lo, hi] the keys' range, key x goes to bucket
// (x - lo) >> s, s chosen so that at most kQsCut / 2 (about n / 2) buckets are
// used -- a monotone map, so the buckets in order are the sorted order up to
// the order inside each bucket.  A histogram, its scan and a scatter by
// shared-memory atomics place the keys by bucket; each thread then sorts its
// buckets by insertion (with s = 0 a bucket holds one key value and needs
// none).  Keys the partition levels leave are near uniform within the
// subarray's range, so buckets hold a few keys; should one hold more than
// kBucketSortMax, the subarray is merge sorted instead (below).  All keys
// equal: nothing to do.
template <typename T>
__device__ __forceinline__ void cta_load_small(const T* __restrict__ keys, uint32_t n, T (&x)[kE]) {
  // coalesced load through L2, every load issued before the first use; the
  // positions past n hold the largest key
  const uint32_t tid = threadIdx.x;
  const T big = (T)~(T)0;
#pragma unroll
  for (uint32_t m = 0; m < kE; m++) {
    const uint32_t i = tid + m * kQsSortThreads;
    if constexpr (sizeof(T) == 8)
      x[m] = i < n ? (T)__ldcg(reinterpret_cast<const unsigned long long*>(keys + i)) : big;
    else
      x[m] = i < n ? (T)__ldcg(reinterpret_cast<const unsigned int*>(keys + i)) : big;
  }
}

// The bucket sort of keys[0..n) (2 <= n <= kQsCut) held in x as
// cta_load_small leaves them.  Returns true (CTA-uniform) once keys[0..n) is
// sorted, false -- keys untouched -- when a bucket holds more than
// kBucketSortMax keys (the merge sort's case).  Ends with a CTA barrier.
template <typename T>
__device__ __forceinline__ bool cta_bucket_sort(T* __restrict__ keys, uint32_t n,
                                                const T (&x)[kE], unsigned char* smem) {
  using S = SortSmem<T>;
  T* const buf = reinterpret_cast<T*>(smem);
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const T big = (T)~(T)0;
  T kmin = big, kmax = 0;
#pragma unroll
  for (uint32_t m = 0; m < kE; m++) {
    if (tid + m * kQsSortThreads < n) {
      kmin = x[m] < kmin ? x[m] : kmin;
      kmax = x[m] > kmax ? x[m] : kmax;
    }
  }
  {  // the CTA's range
#pragma unroll
    for (uint32_t o = 16; o > 0; o >>= 1) {
      const T a = shfl_xor_key(kmin, o), b = shfl_xor_key(kmax, o);
      kmin = a < kmin ? a : kmin;
      kmax = b > kmax ? b : kmax;
    }
    T* red = reinterpret_cast<T*>(smem + S::kRedOff);
    if (lane == 0) {
      red[warp] = kmin;
      red[kQsSortThreads / 32 + warp] = kmax;
    }
    __syncthreads();
#pragma unroll
    for (uint32_t w = 0; w < kQsSortThreads / 32; w++) {
      const T a = red[w], b = red[kQsSortThreads / 32 + w];
      kmin = a < kmin ? a : kmin;
      kmax = b > kmax ? b : kmax;
    }
    __syncthreads();
  }
  if (kmin == kmax) return true;  // all keys equal (the barrier above ends the call)
  const T range = kmax - kmin;
  const uint32_t bits = sizeof(T) == 8 ? 64u - (uint32_t)__clzll((long long)range)
                                       : 32u - (uint32_t)__clz((int)range);
  const uint32_t ln = 32u - (uint32_t)__clz((int)(n - 1));  // ceil(log2 n), n >= 2
  const uint32_t lb = ln > 1 ? ln - 1 : 1;                  // log2 of the bucket count
  const uint32_t sh = bits > lb ? bits - lb : 0u;
  const uint32_t nb = (uint32_t)(range >> sh) + 1;          // buckets in use, <= 2^lb
  uint32_t* const start = reinterpret_cast<uint32_t*>(smem + S::kStartOff);
  uint32_t* const fill = reinterpret_cast<uint32_t*>(smem + S::kFillOff);
  uint32_t* const ws = reinterpret_cast<uint32_t*>(smem + S::kRedOff);
  for (uint32_t b = tid; b < nb; b += kQsSortThreads) start[b] = 0u;
  __syncthreads();
#pragma unroll
  for (uint32_t m = 0; m < kE; m++)
    if (tid + m * kQsSortThreads < n) atomicAdd(&start[(uint32_t)((x[m] - kmin) >> sh)], 1u);
  __syncthreads();
  {  // starts of the buckets: each thread scans a contiguous run of them
    const uint32_t per = (nb + kQsSortThreads - 1) / kQsSortThreads;
    const uint32_t b0 = min(nb, tid * per), b1 = min(nb, b0 + per);
    uint32_t sum = 0, mx = 0;
    for (uint32_t b = b0; b < b1; b++) {
      const uint32_t c = start[b];
      sum += c;
      mx = c > mx ? c : mx;
    }
#pragma unroll
    for (uint32_t o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    uint32_t total = 0;
    uint32_t run = cta_scan_u32(sum, ws, &total);
    for (uint32_t b = b0; b < b1; b++) {
      const uint32_t c = start[b];
      start[b] = run;
      fill[b] = run;
      run += c;
    }
    __syncthreads();
    if (lane == 0) ws[warp] = mx;
    __syncthreads();
    mx = 0;
    for (uint32_t w = 0; w < kQsSortThreads / 32; w++) mx = max(mx, ws[w]);
    if (tid == 0) start[nb] = n;
    if (sh == 0 || mx <= kBucketSortMax) {  // CTA-uniform
      __syncthreads();
#pragma unroll
      for (uint32_t m = 0; m < kE; m++) {
        if (tid + m * kQsSortThreads < n) {
          const uint32_t b = (uint32_t)((x[m] - kmin) >> sh);
          buf[atomicAdd(&fill[b], 1u)] = x[m];
        }
      }
      __syncthreads();
      if (sh > 0) {
        for (uint32_t b = tid; b < nb; b += kQsSortThreads) {
          const uint32_t q0 = start[b], q1 = start[b + 1];
          for (uint32_t p = q0 + 1; p < q1; p++) {
            const T v = buf[p];
            uint32_t q = p;
            while (q > q0 && buf[q - 1] > v) {
              buf[q] = buf[q - 1];
              q--;
            }
            buf[q] = v;
          }
        }
        __syncthreads();
      }
#pragma unroll
      for (uint32_t m = 0; m < kE; m++) {
        const uint32_t i = tid + m * kQsSortThreads;
        if (i < n) keys[i] = buf[i];
      }
      __syncthreads();
      return true;
    }
    __syncthreads();  // every thread has decided before the buffer is reused
  }
  return false;
}

// The merge sort of keys[0..n) (2 <= n <= kQsCut) held in x as cta_load_small
// leaves them.  Ends with a CTA barrier.
template <typename T>
__device__ __forceinline__ void cta_merge_sort(T* __restrict__ keys, uint32_t n, const T (&x)[kE],
                                               unsigned char* smem) {
  using S = SortSmem<T>;
  T* const buf = reinterpret_cast<T*>(smem);
  const uint32_t tid = threadIdx.x;
  constexpr uint32_t kRun = 32 * kE;  // keys one warp sorts in registers
  const T big = (T)~(T)0;
  const uint32_t n16 = (n + kE - 1) / kE * kE;
  const uint32_t nrun = (n + kRun - 1) / kRun * kRun;  // whole warps' runs, padded
  const uint32_t d0 = tid * kE;  // this thread's first output position
  const bool on = d0 < n16;
  const bool warp_on = (d0 & ~(kRun - 1)) < nrun;  // this thread's warp holds keys
#pragma unroll
  for (uint32_t m = 0; m < kE; m++) {
    const uint32_t i = tid + m * kQsSortThreads;
    if (i < nrun) buf[S::pad(i)] = x[m];
  }
  __syncthreads();
  T v[kE];
  if (warp_on) {  // warp-uniform: every lane of a warp with keys takes part
#pragma unroll
    for (uint32_t r = 0; r < kE; r++) v[r] = buf[S::pad(d0 + r)];
    sort16(v);
    warp_merge_to_512(v, tid & 31u);
#pragma unroll
    for (uint32_t r = 0; r < kE; r++) buf[S::pad(d0 + r)] = v[r];
  }
  __syncthreads();
  for (uint32_t L = kRun; L < n16; L <<= 1) {
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

// Sorts keys[0..n), n <= kQsCut: the bucket sort, else the merge sort.  Ends
// with a CTA barrier.
template <typename T>
__device__ __forceinline__ void cta_sort_small(T* __restrict__ keys, uint32_t n, unsigned char* smem) {
  if (n < 2) {
    __syncthreads();
    return;
  }
  T x[kE];
  cta_load_small<T>(keys, n, x);
  if (!cta_bucket_sort<T>(keys, n, x, smem)) cta_merge_sort<T>(keys, n, x, smem);
}

}  // namespace lp
