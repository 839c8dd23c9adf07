// lp_qs.cu -- kernels of the quicksort on the partition (records and the
// level rule in lp_qs.cuh): segment records with median-of-3 pivots, the
// children split, and the shared-memory sort of subarrays of at most kQsCut
// keys.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lp_batch_init.cuh"
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

// One level's set-up of one slice in one launch: the job record to the device
// (the level's later kernels read it there), the level counts reset (first
// slice), and every item's segment record built with its engine state, in
// place of the batched engine's own set-up launch.
template <typename T>
__global__ void qs_level_start_kernel(const QsJob J, QsJob* d_job, SegDesc* segs,
                                      uint64_t batch_seed, unsigned long long* traffic,
                                      unsigned long long* tround, uint32_t* bar,
                                      uint32_t reset_counts) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    *d_job = J;
    if (reset_counts) *J.lc = QsLevelCounts{0u, 0u, 0u, 0u};
  }
  batch_launch_reset(traffic, tround, bar, i);
  if (i >= J.count) return;
  SegDesc d = qs_item_record<T>(static_cast<T*>(J.keys), J.items[i], J.seed, J.level, J.samples);
  batch_seg_init<T>(d, batch_seed);
  segs[J.seg_base + i] = d;
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

// The bucket sort of every small subarray; those whose keys bunch go to the
// job's merge list.  Without the merge sort's code the kernel fits 64
// registers a thread: 4 CTAs per SM keep more subarrays' loads in flight than
// 3 did with both sorts in one kernel.
template <typename T>
__global__ void __launch_bounds__(kQsSortThreads, 4) qs_small_sort_kernel(const QsJob* jobs) {
  extern __shared__ __align__(16) unsigned char qs_smem[];
  const QsJob& J = jobs[blockIdx.y];
  const uint32_t cnt = *reinterpret_cast<volatile uint32_t*>(&J.lc->small);
  T* keys = static_cast<T*>(J.keys);
  for (uint32_t s = blockIdx.x; s < cnt; s += gridDim.x) {
    const QsSmall q = J.small[s];
    const uint32_t n = (uint32_t)q.n;
    if (n < 2) continue;
    T x[kE];
    cta_load_small<T>(keys + q.lo, n, x);
    if (!cta_bucket_sort<T>(keys + q.lo, n, x, qs_smem) && threadIdx.x == 0)
      J.merge[atomicAdd(&J.lc->merge, 1u)] = s;
  }
}

// The merge sort of the subarrays the bucket sort listed.
template <typename T>
__global__ void __launch_bounds__(kQsSortThreads, 3) qs_merge_sort_kernel(const QsJob* jobs) {
  extern __shared__ __align__(16) unsigned char qs_smem[];
  const QsJob& J = jobs[blockIdx.y];
  const uint32_t cnt = *reinterpret_cast<volatile uint32_t*>(&J.lc->merge);
  T* keys = static_cast<T*>(J.keys);
  for (uint32_t k = blockIdx.x; k < cnt; k += gridDim.x) {
    const QsSmall q = J.small[J.merge[k]];
    T x[kE];
    cta_load_small<T>(keys + q.lo, (uint32_t)q.n, x);
    cta_merge_sort<T>(keys + q.lo, (uint32_t)q.n, x, qs_smem);
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

template <typename T>
cudaError_t launch_qs_level_start(const QsJob& J, QsJob* d_job, SegDesc* segs,
                                  uint64_t batch_seed, const BatchScratch& B, bool reset_counts,
                                  cudaStream_t st) {
  const uint32_t threads = J.count > kBatchRoundSlots * 4 ? J.count : kBatchRoundSlots * 4;
  qs_level_start_kernel<T><<<(threads + 255) / 256, 256, 0, st>>>(
      J, d_job, segs, batch_seed, B.totals + 2, B.tround, B.bar, reset_counts ? 1u : 0u);
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
  qs_small_sort_kernel<T><<<dim3(ctas, njobs), kQsSortThreads, SortSmem<T>::kBucketBytes, st>>>(
      jobs);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_qs_merge_sort(const QsJob* jobs, uint32_t njobs, uint32_t ctas,
                                 cudaStream_t st) {
  if (njobs == 0 || ctas == 0) return cudaSuccess;
  qs_merge_sort_kernel<T><<<dim3(ctas, njobs), kQsSortThreads, SortSmem<T>::kMergeBytes, st>>>(
      jobs);
  return cudaGetLastError();
}

cudaError_t qs_prepare() {
  cudaError_t e = cudaFuncSetAttribute(qs_small_sort_kernel<uint64_t>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SortSmem<uint64_t>::kBucketBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(qs_small_sort_kernel<uint32_t>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SortSmem<uint32_t>::kBucketBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(qs_merge_sort_kernel<uint64_t>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SortSmem<uint64_t>::kMergeBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(qs_merge_sort_kernel<uint32_t>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SortSmem<uint32_t>::kMergeBytes);
  return e;
}

template cudaError_t launch_qs_build<uint64_t>(const QsJob*, uint32_t, uint32_t, SegDesc*,
                                               cudaStream_t);
template cudaError_t launch_qs_build<uint32_t>(const QsJob*, uint32_t, uint32_t, SegDesc*,
                                               cudaStream_t);
template cudaError_t launch_qs_level_start<uint64_t>(const QsJob&, QsJob*, SegDesc*, uint64_t,
                                                     const BatchScratch&, bool, cudaStream_t);
template cudaError_t launch_qs_level_start<uint32_t>(const QsJob&, QsJob*, SegDesc*, uint64_t,
                                                     const BatchScratch&, bool, cudaStream_t);
template cudaError_t launch_qs_small_sort<uint64_t>(const QsJob*, uint32_t, uint32_t,
                                                    cudaStream_t);
template cudaError_t launch_qs_small_sort<uint32_t>(const QsJob*, uint32_t, uint32_t,
                                                    cudaStream_t);
template cudaError_t launch_qs_merge_sort<uint64_t>(const QsJob*, uint32_t, uint32_t,
                                                    cudaStream_t);
template cudaError_t launch_qs_merge_sort<uint32_t>(const QsJob*, uint32_t, uint32_t,
                                                    cudaStream_t);

}  // namespace lp
