// lp_qs.cu -- kernels of the quicksort on the partition (records and the
// level rule in lp_qs.cuh): segment records with median-of-3 pivots, the
// children split, and the shared-memory sort of subarrays of at most kQsCut
// keys.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lp_qs.cuh"

namespace lp {

namespace {

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

__device__ __forceinline__ void qs_push(const QsJob& J, uint64_t lo, uint64_t n) {
  if (n <= 1) return;  // a single key is in place
  if (n <= kQsCut) {
    J.small[atomicAdd(&J.lc->small, 1u)] = QsSmall{lo, n};
    atomicAdd(J.sort_keys, (unsigned long long)n);
  } else {
    J.next[atomicAdd(&J.lc->next, 1u)] = QsItem{lo, n, 0, 0};
  }
}

__global__ void qs_split_kernel(const QsJob* jobs, const SegDesc* segs, const uint64_t* splits,
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

// ---------------------------------------------------------------- small sort
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

template <typename T>
__global__ void __launch_bounds__(kQsSortThreads, 4) qs_small_sort_kernel(const QsJob* jobs) {
  using S = SortSmem<T>;
  extern __shared__ __align__(16) unsigned char qs_smem[];
  T* const buf = reinterpret_cast<T*>(qs_smem);
  const QsJob& J = jobs[blockIdx.y];
  const uint32_t tid = threadIdx.x;
  const uint32_t cnt = *reinterpret_cast<volatile uint32_t*>(&J.lc->small);
  T* keys = static_cast<T*>(J.keys);
  const T big = (T)~(T)0;
  for (uint32_t s = blockIdx.x; s < cnt; s += gridDim.x) {
    const QsSmall q = J.small[s];
    const uint32_t n = (uint32_t)q.n;
    const uint32_t n16 = (n + kE - 1) / kE * kE;
    const uint32_t d0 = tid * kE;  // this thread's first output position
    const bool on = d0 < n16;
    {  // coalesced load, every load issued before the first store
      T x[kE];
#pragma unroll
      for (uint32_t m = 0; m < kE; m++) {
        const uint32_t i = tid + m * kQsSortThreads;
        x[m] = i < n ? keys[q.lo + i] : big;
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
      if (i < n) keys[q.lo + i] = buf[S::pad(i)];
    }
    __syncthreads();
  }
}

}  // namespace

template <typename T>
cudaError_t launch_qs_build(const QsJob* jobs, uint32_t njobs, uint32_t max_count, SegDesc* segs,
                            cudaStream_t st) {
  if (njobs == 0 || max_count == 0) return cudaSuccess;
  qs_build_kernel<T><<<dim3((max_count + 255) / 256, njobs), 256, 0, st>>>(jobs, segs);
  return cudaGetLastError();
}

cudaError_t launch_qs_split(const QsJob* jobs, uint32_t njobs, uint32_t max_count,
                            const SegDesc* segs, const uint64_t* splits,
                            const unsigned long long* traffic, unsigned long long* traffic_acc,
                            cudaStream_t st) {
  if (njobs == 0) return cudaSuccess;
  const uint32_t gx = max_count ? (max_count + 255) / 256 : 1;
  qs_split_kernel<<<dim3(gx, njobs), 256, 0, st>>>(jobs, segs, splits, traffic, traffic_acc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_qs_small_sort(const QsJob* jobs, uint32_t njobs, uint32_t ctas,
                                 cudaStream_t st) {
  if (njobs == 0 || ctas == 0) return cudaSuccess;
  qs_small_sort_kernel<T><<<dim3(ctas, njobs), kQsSortThreads, SortSmem<T>::kBytes, st>>>(jobs);
  return cudaGetLastError();
}

cudaError_t qs_prepare() {
  cudaError_t e = cudaFuncSetAttribute(qs_small_sort_kernel<uint64_t>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SortSmem<uint64_t>::kBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(qs_small_sort_kernel<uint32_t>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SortSmem<uint32_t>::kBytes);
  return e;
}

template cudaError_t launch_qs_build<uint64_t>(const QsJob*, uint32_t, uint32_t, SegDesc*,
                                               cudaStream_t);
template cudaError_t launch_qs_build<uint32_t>(const QsJob*, uint32_t, uint32_t, SegDesc*,
                                               cudaStream_t);
template cudaError_t launch_qs_small_sort<uint64_t>(const QsJob*, uint32_t, uint32_t,
                                                    cudaStream_t);
template cudaError_t launch_qs_small_sort<uint32_t>(const QsJob*, uint32_t, uint32_t,
                                                    cudaStream_t);

}  // namespace lp
