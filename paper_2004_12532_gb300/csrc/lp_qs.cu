// lp_qs.cu -- kernels of the quicksort on the partition (records and the
// level rule in lp_qs.cuh): segment records with median-of-3 pivots, the
// children split, and the shared-memory sort of subarrays of at most kQsCut
// keys.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lp_qs.cuh"
#include "lp_qs_pivot.cuh"
#include "lp_qs_sort.cuh"

namespace lp {

namespace {

// Segment records of every job slice: blockIdx.y = job, x = item.
template <typename T>
__global__ void qs_build_kernel(const QsJob* jobs, SegDesc* segs) {
  const QsJob& J = jobs[blockIdx.y];
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= J.count) return;
  const QsItem q = J.items[i];
  T* keys = static_cast<T*>(J.keys);
  const uint64_t h = qs_item_hash(J.seed, J.level, q.lo, q.n);
  SegDesc d = {};
  d.keys = keys + q.lo;
  d.n = q.n;
  if (q.eq) {
    d.pivot = q.pivot - 1;  // q.pivot > 0: a zero pivot never makes an equal-key item
  } else {
    d.pivot = (uint64_t)(J.samples == kQsSamplesMax ? qs_median<kQsSamplesMax>(keys, q.lo, q.n, h)
                                                    : qs_median<3>(keys, q.lo, q.n, h));
  }
  // the subarray and level name it, not its place in the list
  d.salt = sm_stream(h, kQsSamplesMax + 1);
  segs[J.seg_base + i] = d;
}

__device__ __forceinline__ void qs_push(const QsJob& J, uint64_t lo, uint64_t n) {
  if (n <= 1) return;  // a single key is in place
  if (n <= (J.local_cut ? (uint64_t)J.local_cut : kQsCut)) {
    J.small[atomicAdd(&J.lc->small, 1u)] = QsSmall{lo, n, J.level + 1, 0u};
    atomicAdd(J.sort_keys, (unsigned long long)n);
  } else {
    J.next[atomicAdd(&J.lc->next, 1u)] = QsItem{lo, n, 0, 0};
    atomicMax(&J.lc->max_next, n < 0xffffffffull ? (uint32_t)n : 0xffffffffu);
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
    if (p != 0) {
      J.next[atomicAdd(&J.lc->next, 1u)] = QsItem{q.lo, q.n, p, 1};
      atomicMax(&J.lc->max_next, q.n < 0xffffffffull ? (uint32_t)q.n : 0xffffffffu);
    }
    return;
  }
  qs_push(J, q.lo, t);
  qs_push(J, q.lo + t, q.n - t);
}

template <typename T>
__global__ void __launch_bounds__(kQsSortThreads, 3) qs_small_sort_kernel(const QsJob* jobs) {
  extern __shared__ __align__(16) unsigned char qs_smem[];
  const QsJob& J = jobs[blockIdx.y];
  const uint32_t cnt = *reinterpret_cast<volatile uint32_t*>(&J.lc->small);
  T* keys = static_cast<T*>(J.keys);
  for (uint32_t s = blockIdx.x; s < cnt; s += gridDim.x) {
    const QsSmall q = J.small[s];
    cta_sort_small<T>(keys + q.lo, (uint32_t)q.n, qs_smem);
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
