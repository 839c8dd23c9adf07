// lp_qs.cu -- kernels of the quicksort on the partition (records and the
// level rule in lp_qs.cuh): segment records with median-of-3 pivots, the
// children split, and the shared-memory sort of subarrays of at most kQsCut
// keys.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lp_qs.cuh"
#include "lp_qs_level.cuh"
#include "lp_qs_sort.cuh"

namespace lp {

namespace {

// Segment records of every job slice: blockIdx.y = job, x = item.
template <typename T>
__global__ void qs_build_kernel(const QsJob* jobs, SegDesc* segs) {
  const QsJob& J = jobs[blockIdx.y];
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= J.count) return;
  segs[J.seg_base + i] =
      qs_item_record<T>(static_cast<T*>(J.keys), J.items[i], J.seed, J.level, J.samples);
}

__global__ void qs_split_kernel(const QsJob* jobs, const SegDesc* segs, const uint64_t* splits,
                                const unsigned long long* traffic,
                                unsigned long long* traffic_acc) {
  const QsJob& J = jobs[blockIdx.y];
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *traffic_acc += *traffic;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= J.count) return;
  qs_item_children(J, J.items[i], splits[J.seg_base + i], segs[J.seg_base + i].pivot);
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
