// lp_quicksort.cu -- quicksort of one array on the partition (Sec. 5, "A Full
// Quicksort"): the paper partitions in parallel at the top levels and
// serially once subproblems are small.  Here every level partitions all open
// subarrays of the array at once through the batched engine (lp_batched.cu)
// and the subarrays of at most kQsCut keys are sorted by one CTA each in
// shared memory (kernels in lp_qs.cuh).
//
// Per level: build the segment records (median-of-3 or -15 pivots), one batched
// launch per slice of at most kSlice subarrays, split into children, sort the
// level's small subarrays, read the next list's size back (one host
// synchronisation per level), and merge sort the small subarrays the bucket
// sort turned down, if it turned any down.  Auxiliary memory: two item lists
// of at most n / (kQsCut + 1) items (32 bytes each), a small list of twice
// that (16 bytes each) with a merge list beside it (4 bytes each), and the
// records of one slice of at most kSlice items (about 2.9 MB) -- about 0.4%
// of a uint64 array's bytes at n = 2^28.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lp_batched.h"
#include "lp_qs.cuh"

namespace lp {

namespace {

constexpr uint32_t kSlice = 16384;  // segments per batched launch, at most
constexpr uint32_t kMaxSortLevels = 4096;


struct QsLayout {
  QsItem* lists[2];
  QsSmall* small;
  uint32_t* merge;
  SegDesc* segs;
  uint64_t* splits;
  QsJob* jobs;                      // one record per slice
  QsLevelCounts* lc;
  unsigned long long* acc;          // [0] keys streamed by partitions, [1] keys sorted,
                                    // [2..6] the tail kernel's tallies (launch_qs_local)
  void* batch;
  uint64_t maxseg;
  uint32_t slice, max_slices;
  size_t bytes;
};

QsLayout qs_layout(void* base, uint64_t n) {
  QsLayout L{};
  L.maxseg = n / (kQsCut + 1) + 1;
  L.slice = (uint32_t)(L.maxseg < kSlice ? L.maxseg : kSlice);
  L.max_slices = (uint32_t)((L.maxseg + L.slice - 1) / L.slice);
  unsigned char* p = static_cast<unsigned char*>(base);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* r = p ? p + off : nullptr;
    off += (bytes + 255) / 256 * 256;
    return r;
  };
  L.lists[0] = reinterpret_cast<QsItem*>(take(L.maxseg * sizeof(QsItem)));
  L.lists[1] = reinterpret_cast<QsItem*>(take(L.maxseg * sizeof(QsItem)));
  L.small = reinterpret_cast<QsSmall*>(take(2 * L.maxseg * sizeof(QsSmall)));
  L.merge = reinterpret_cast<uint32_t*>(take(2 * L.maxseg * sizeof(uint32_t)));
  L.segs = reinterpret_cast<SegDesc*>(take((size_t)L.slice * sizeof(SegDesc)));
  L.splits = reinterpret_cast<uint64_t*>(take((size_t)L.slice * 8));
  L.jobs = reinterpret_cast<QsJob*>(take((size_t)L.max_slices * sizeof(QsJob)));
  L.lc = reinterpret_cast<QsLevelCounts*>(take(sizeof(QsLevelCounts)));
  L.acc = reinterpret_cast<unsigned long long*>(take(64));
  L.batch = take(batch_scratch_bytes(L.slice));
  L.bytes = off;
  return L;
}

}  // namespace

size_t quicksort_scratch_bytes(uint64_t n) { return qs_layout(nullptr, n).bytes; }
size_t quicksort_staging_bytes(uint64_t n) {
  return (size_t)qs_layout(nullptr, n).max_slices * sizeof(QsJob) + 64;
}

template <typename T>
cudaError_t launch_quicksort(T* keys, uint64_t n, uint64_t seed, uint32_t samples, void* scratch,
                             void* staging, const BatchTuning& tune, uint32_t* bar,
                             uint32_t* status, LaunchCfg& cfg, const cudaEvent_t* ev,
                             SortStats* stats) {
  cudaStream_t st = cfg.stream;
  *stats = SortStats{};
  if (n < 2) return cudaSuccess;
  const QsLayout L = qs_layout(scratch, n);
  const BatchScratch Bs = carve_batch_scratch(L.batch, L.slice, bar, status);
  QsJob* hjobs = static_cast<QsJob*>(staging);
  unsigned char* hback = static_cast<unsigned char*>(staging) + L.max_slices * sizeof(QsJob);
  const uint64_t batch_seed = sm_stream(seed, 0x51);
  int dev = 0;
  uint32_t tail_grid = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = qs_local_grid<T>(dev, &tail_grid);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.acc, 0, 64, st);
  if (e != cudaSuccess) return e;
  // the first level: the whole array as one item, or as the only small subarray
  uint64_t open = 0;
  if (n > kQsCut) {
    const QsItem whole{0, n, 0, 0};
    e = cudaMemcpyAsync(L.lists[0], &whole, sizeof(whole), cudaMemcpyHostToDevice, st);
    open = 1;
  } else {
    const QsSmall whole{0, (uint32_t)n, 0u};
    e = cudaMemcpyAsync(L.small, &whole, sizeof(whole), cudaMemcpyHostToDevice, st);
  }
  if (e != cudaSuccess) return e;
  const QsLevelCounts first{0, n > kQsCut ? 0u : 1u, 0u, 0u};
  e = cudaMemcpyAsync(L.lc, &first, sizeof(first), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  auto mark = [&](int k) -> cudaError_t { return ev ? cudaEventRecord(ev[k], st) : cudaSuccess; };
  auto elapsed = [&](int a, int b, float* acc) {
    float ms = 0.f;
    if (ev && cudaEventElapsedTime(&ms, ev[a], ev[b]) == cudaSuccess) *acc += ms;
  };
  uint32_t cur = 0, levels = 0;
  uint64_t peak_open = open;
  for (;;) {
    // one record per slice of the level's list (one record, of no items,
    // for the small-only first level: the small sort reads its lists)
    const uint32_t nslices = (uint32_t)((open + L.slice - 1) / L.slice);
    const uint32_t nrec = nslices ? nslices : 1;
    for (uint32_t k = 0; k < nrec; k++) {
      const uint64_t o = (uint64_t)k * L.slice;
      QsJob& J = hjobs[k];
      J.keys = keys;
      J.items = L.lists[cur] + o;
      J.next = L.lists[cur ^ 1];
      J.small = L.small;
      J.merge = L.merge;
      J.lc = L.lc;
      J.sort_keys = L.acc + 1;
      J.seed = seed;
      J.level = levels;
      J.count = (uint32_t)(open > o ? (open - o < L.slice ? open - o : L.slice) : 0);
      J.seg_base = 0;
      J.samples = samples;
      J.local_cut = 0;
    }
    // a level with items: each slice's first launch writes its job record,
    // resets the level counts (first slice) and sets up the records -- one
    // launch before the persistent one, where a copy, a reset and two
    // set-up kernels would each wait for the host to issue them
    if (nslices == 0) {  // the small-only first level: its record for the sort
      e = cudaMemcpyAsync(L.jobs, hjobs, sizeof(QsJob), cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return e;
    }
    if ((e = mark(0)) != cudaSuccess) return e;
    for (uint32_t k = 0; k < nslices; k++) {
      const uint32_t cnt = hjobs[k].count;
      e = launch_qs_level_start<T>(hjobs[k], L.jobs + k, L.segs, batch_seed, Bs, k == 0, st);
      if (e != cudaSuccess) return e;
      cfg.launches++;
      e = launch_batched<T>(L.segs, cnt, batch_seed, L.splits, Bs, tune, cfg, true);
      if (e != cudaSuccess) return e;
      e = launch_qs_split(L.jobs + k, 1, cnt, L.segs, L.splits, Bs.totals + 2, L.acc, st);
      if (e != cudaSuccess) return e;
      cfg.launches++;
    }
    if ((e = mark(1)) != cudaSuccess) return e;
    // the level's small subarrays (at most two per item; the count is read on the device)
    const uint64_t small_bound = open ? 2 * open : 1;
    e = launch_qs_small_sort<T>(L.jobs, 1, (uint32_t)(small_bound < 8192 ? small_bound : 8192),
                                st);
    if (e != cudaSuccess) return e;
    cfg.launches++;
    if ((e = mark(2)) != cudaSuccess) return e;
    e = cudaMemcpyAsync(hback, L.lc, sizeof(QsLevelCounts), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    elapsed(0, 1, &stats->partition_ms);
    elapsed(1, 2, &stats->sort_ms);
    const uint32_t merges = reinterpret_cast<const QsLevelCounts*>(hback)->merge;
    if (merges > 0) {  // before the next level reuses the lists
      if ((e = mark(1)) != cudaSuccess) return e;
      e = launch_qs_merge_sort<T>(L.jobs, 1, merges < 2048 ? merges : 2048, st);
      if (e != cudaSuccess) return e;
      cfg.launches++;
      if ((e = mark(2)) != cudaSuccess) return e;
      if (ev && (e = cudaEventSynchronize(ev[2])) != cudaSuccess) return e;
      elapsed(1, 2, &stats->sort_ms);
    }
    if (nslices == 0) break;  // the small-only first level is done
    levels++;
    open = reinterpret_cast<const QsLevelCounts*>(hback)->next;
    const uint64_t max_item = reinterpret_cast<const QsLevelCounts*>(hback)->max_next;
    cur ^= 1;
    if (open == 0) break;
    if (levels > kMaxSortLevels) return cudaErrorUnknown;  // sizes shrink every level
    if (open > peak_open) peak_open = open;
    if (qs_is_tail(open, peak_open, max_item)) {  // the tail, in one launch
      if ((e = mark(1)) != cudaSuccess) return e;
      e = launch_qs_local<T>(keys, L.lists[cur], (uint32_t)open, levels, seed, samples,
                             L.acc + 2, status, tail_grid, st);
      if (e != cudaSuccess) return e;
      cfg.launches += 2;  // counter reset + kernel
      if ((e = mark(2)) != cudaSuccess) return e;
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
      elapsed(1, 2, &stats->tail_ms);
      stats->tail_items = (uint32_t)open;
      break;
    }
  }
  e = cudaMemcpyAsync(hback, L.acc, 56, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  const unsigned long long* acc = reinterpret_cast<const unsigned long long*>(hback);
  stats->levels = levels;
  stats->partition_keys = acc[0];
  stats->sort_keys = acc[1] + acc[3] + (n <= kQsCut ? n : 0);
  stats->tail_keys = acc[2];
  return cudaGetLastError();
}

template cudaError_t launch_quicksort<uint64_t>(uint64_t*, uint64_t, uint64_t, uint32_t, void*,
                                                void*, const BatchTuning&, uint32_t*, uint32_t*,
                                                LaunchCfg&, const cudaEvent_t*, SortStats*);
template cudaError_t launch_quicksort<uint32_t>(uint32_t*, uint64_t, uint64_t, uint32_t, void*,
                                                void*, const BatchTuning&, uint32_t*, uint32_t*,
                                                LaunchCfg&, const cudaEvent_t*, SortStats*);

}  // namespace lp
