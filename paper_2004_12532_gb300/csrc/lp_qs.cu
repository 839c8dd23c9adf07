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
// One CTA sorts one subarray of n <= kQsCut keys: P = the next power of two
// (at least 8), padded with the largest key.  Thread t owns the 8 keys
// [8t, 8t + 8): it sorts them with a 19-comparator network, then log2(P / 8)
// merge passes double the sorted runs; in each, thread t finds where output
// position 8t of its merged pair of runs splits the two inputs (a binary
// search along the merge-path diagonal) and merges its 8 outputs.  Runs live
// in shared memory, two buffers in turn, padded by one word every 128 bytes so
// that the threads' 8-key blocks fall in distinct banks.
constexpr uint32_t kE = 8;
static_assert(kQsSortThreads * kE == kQsCut, "one CTA holds a whole small subarray");

template <typename T>
struct SortSmem {
  static constexpr uint32_t kShift = sizeof(T) == 8 ? 4 : 5;  // words per 128 bytes
  static constexpr uint32_t kWords = kQsCut + (kQsCut >> kShift);
  static constexpr size_t kBytes = 2 * kWords * sizeof(T);
  __device__ static __forceinline__ uint32_t pad(uint32_t i) { return i + (i >> kShift); }
};

template <typename T>
__device__ __forceinline__ void cswap(T& a, T& b) {
  const bool s = b < a;
  const T x = s ? b : a, y = s ? a : b;
  a = x;
  b = y;
}

template <typename T>
__device__ __forceinline__ void sort8(T (&v)[kE]) {
  cswap(v[0], v[2]); cswap(v[1], v[3]); cswap(v[4], v[6]); cswap(v[5], v[7]);
  cswap(v[0], v[4]); cswap(v[1], v[5]); cswap(v[2], v[6]); cswap(v[3], v[7]);
  cswap(v[0], v[1]); cswap(v[2], v[3]); cswap(v[4], v[5]); cswap(v[6], v[7]);
  cswap(v[2], v[4]); cswap(v[3], v[5]);
  cswap(v[1], v[4]); cswap(v[3], v[6]);
  cswap(v[1], v[2]); cswap(v[3], v[4]); cswap(v[5], v[6]);
}

template <typename T>
__global__ void __launch_bounds__(kQsSortThreads) qs_small_sort_kernel(const QsJob* jobs) {
  using S = SortSmem<T>;
  extern __shared__ __align__(16) unsigned char qs_smem[];
  T* const buf0 = reinterpret_cast<T*>(qs_smem);  // two buffers of S::kWords words
  const QsJob& J = jobs[blockIdx.y];
  const uint32_t tid = threadIdx.x;
  const uint32_t cnt = *reinterpret_cast<volatile uint32_t*>(&J.lc->small);
  T* keys = static_cast<T*>(J.keys);
  const T big = (T)~(T)0;
  for (uint32_t s = blockIdx.x; s < cnt; s += gridDim.x) {
    const QsSmall q = J.small[s];
    const uint32_t n = (uint32_t)q.n;
    uint32_t P = kE;
    while (P < n) P <<= 1;
    const uint32_t d0 = tid * kE;  // this thread's first output position
    const bool on = d0 < P;
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
        if (i < P) buf0[S::pad(i)] = x[m];
      }
    }
    __syncthreads();
    T v[kE];
    if (on) {
#pragma unroll
      for (uint32_t r = 0; r < kE; r++) v[r] = buf0[S::pad(d0 + r)];
      sort8(v);
#pragma unroll
      for (uint32_t r = 0; r < kE; r++) buf0[S::pad(d0 + r)] = v[r];
    }
    __syncthreads();
    uint32_t cur = 0;
    for (uint32_t L = kE; L < P; L <<= 1) {
      const T* src = buf0 + cur * S::kWords;
      T* dst = buf0 + (cur ^ 1) * S::kWords;
      if (on) {
        const uint32_t base = d0 & ~(2 * L - 1), d = d0 - base;
        const uint32_t ab = base, bb = base + L;
        uint32_t lo = d > L ? d - L : 0, hi = d < L ? d : L;
        while (lo < hi) {  // the merge-path split of diagonal d
          const uint32_t mid = (lo + hi) >> 1;
          if (src[S::pad(ab + mid)] <= src[S::pad(bb + d - 1 - mid)]) lo = mid + 1;
          else hi = mid;
        }
        uint32_t i = lo, j = d - lo;
        T a = i < L ? src[S::pad(ab + i)] : big;
        T b = j < L ? src[S::pad(bb + j)] : big;
#pragma unroll
        for (uint32_t r = 0; r < kE; r++) {
          const bool ta = j >= L || (i < L && a <= b);
          v[r] = ta ? a : b;
          i += ta ? 1u : 0u;
          j += ta ? 0u : 1u;
          const uint32_t ni = ta ? i : j;
          if (ni < L) {
            const T nx = src[S::pad((ta ? ab : bb) + ni)];
            if (ta) a = nx; else b = nx;
          }
        }
#pragma unroll
        for (uint32_t r = 0; r < kE; r++) dst[S::pad(d0 + r)] = v[r];
      }
      __syncthreads();
      cur ^= 1;
    }
#pragma unroll
    for (uint32_t m = 0; m < kE; m++) {
      const uint32_t i = tid + m * kQsSortThreads;
      if (i < n) keys[q.lo + i] = buf0[cur * S::kWords + S::pad(i)];
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
