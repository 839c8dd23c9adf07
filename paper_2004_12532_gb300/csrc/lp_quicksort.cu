// lp_quicksort.cu -- quicksort on the partition (Sec. 5, "A Full Quicksort"):
// the paper partitions in parallel at the top levels and serially once
// subproblems are small.  On the GPU every level partitions all open
// subarrays at once through the batched engine (lp_batched.cu), and
// subarrays of at most kCut keys are sorted by one CTA each in shared memory.
//
// Per level (device-resident lists; the host reads back the list sizes):
//   build   pivot of each open subarray = median of three seeded samples;
//   batch   partition every open subarray by [x <= pivot];
//   split   children [lo, lo+t) and [lo+t, hi); a child of at most kCut keys
//           goes to the level's small list; when every key was <= pivot
//           (t = n), the subarray is partitioned again by [x < pivot]
//           (pivot - 1) and only [lo, lo+t') stays open -- the keys equal to
//           the pivot are in final place;
//   sort    every subarray of the small list is sorted in shared memory.
// Every open subarray holds more than kCut keys, so a level has at most
// n / (kCut + 1) of them: the lists cost < 0.3% of the array's bytes (uint64).
// The batched engine's per-segment records are used in slices of at most
// kSlice segments, so they cost a fixed amount whatever n is.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lp_batched.h"
#include "lp_device.cuh"
#include "lp_launch.h"
#include "lp_plan.h"

namespace lp {

namespace {

constexpr uint64_t kCut = 4096;     // subarrays this small are sorted in shared memory
constexpr uint32_t kSlice = 16384;  // segments per batched launch, at most
constexpr uint32_t kMaxSortLevels = 4096;

struct QsSeg {
  uint64_t lo, n;
};
struct QsEq {
  uint64_t lo, n, pivot;
};

// list sizes of the level and keys streamed, in device memory
struct QsCounts {
  uint32_t next, small, eq, pad;           // reset every level
  unsigned long long part_keys, sort_keys; // whole call
};

template <typename T>
__device__ __forceinline__ T ldk(const T* p) {
  if constexpr (sizeof(T) == 8) return (T)__ldcg(reinterpret_cast<const unsigned long long*>(p));
  else return (T)__ldcg(reinterpret_cast<const unsigned int*>(p));
}

// Segment records of one slice of the open list: the pivot is the median of
// three keys at seeded positions of the subarray.
template <typename T>
__global__ void qs_build_kernel(const QsSeg* list, uint32_t count, T* keys, uint64_t seed,
                                SegDesc* out) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= count) return;
  const QsSeg q = list[s];
  const uint64_t h = sm_stream(seed, q.lo ^ (q.n << 32));
  const T a = ldk(&keys[q.lo + range_of(sm_stream(h, 0), q.n)]);
  const T b = ldk(&keys[q.lo + range_of(sm_stream(h, 1), q.n)]);
  const T c = ldk(&keys[q.lo + range_of(sm_stream(h, 2), q.n)]);
  const T mx = a > b ? a : b, mn = a > b ? b : a;
  SegDesc d = {};
  d.keys = keys + q.lo;
  d.n = q.n;
  d.pivot = (uint64_t)(c > mx ? mx : (c < mn ? mn : c));
  d.salt = q.lo;  // the subarray's place names it, whatever its place in the list
  out[s] = d;
}

// Segment records of one slice of the equal-key list: partition by [x < pivot].
template <typename T>
__global__ void qs_build_eq_kernel(const QsEq* list, uint32_t count, T* keys, SegDesc* out) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= count) return;
  const QsEq q = list[s];
  SegDesc d = {};
  d.keys = keys + q.lo;
  d.n = q.n;
  d.pivot = q.pivot - 1;  // q.pivot > 0 (a zero pivot never reaches this list)
  d.salt = q.lo;
  out[s] = d;
}

__device__ __forceinline__ void qs_push(QsSeg* next, QsSeg* small, QsCounts* c, uint64_t lo,
                                        uint64_t n) {
  if (n <= 1) return;  // a single key is in place
  if (n <= kCut) {
    small[atomicAdd(&c->small, 1u)] = QsSeg{lo, n};
    atomicAdd(&c->sort_keys, (unsigned long long)n);
  } else {
    next[atomicAdd(&c->next, 1u)] = QsSeg{lo, n};
  }
}

// keys the batched launch just before streamed, added to the call's total
__device__ __forceinline__ void qs_add_traffic(QsCounts* c, const unsigned long long* traffic) {
  if (blockIdx.x == 0 && threadIdx.x == 0) c->part_keys += *traffic;
}

// Children of each partitioned subarray.  A subarray with no successor goes
// to the equal-key list unless its pivot is 0 (then every key is 0).
__global__ void qs_split_kernel(const QsSeg* list, uint32_t count, const SegDesc* segs,
                                const uint64_t* splits, QsSeg* next, QsSeg* small, QsEq* eq,
                                QsCounts* c, const unsigned long long* traffic) {
  qs_add_traffic(c, traffic);
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= count) return;
  const QsSeg q = list[s];
  const uint64_t t = splits[s];
  if (t == q.n) {
    const uint64_t pivot = segs[s].pivot;
    if (pivot != 0) eq[atomicAdd(&c->eq, 1u)] = QsEq{q.lo, q.n, pivot};
    return;
  }
  qs_push(next, small, c, q.lo, t);
  qs_push(next, small, c, q.lo + t, q.n - t);
}

// After the pass by [x < pivot]: [lo, lo + t') stays open, the rest is final.
__global__ void qs_split_eq_kernel(const QsEq* eq, uint32_t count, const uint64_t* splits,
                                   QsSeg* next, QsSeg* small, QsCounts* c,
                                   const unsigned long long* traffic) {
  qs_add_traffic(c, traffic);
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= count) return;
  qs_push(next, small, c, eq[s].lo, splits[s]);
}

// One CTA sorts one subarray of at most kCut keys: bitonic sorting network in
// shared memory over the next power of two, padded with the largest key.
constexpr uint32_t kSortThreads = 512;

template <typename T>
__global__ void __launch_bounds__(kSortThreads) qs_small_sort_kernel(const QsSeg* small,
                                                                     uint32_t count, T* keys) {
  __shared__ T buf[kCut];
  const uint32_t tid = threadIdx.x;
  for (uint32_t s = blockIdx.x; s < count; s += gridDim.x) {
    const QsSeg q = small[s];
    const uint32_t n = (uint32_t)q.n;
    uint32_t P = 2;
    while (P < n) P <<= 1;
    for (uint32_t i = tid; i < P; i += kSortThreads)
      buf[i] = i < n ? ldk(&keys[q.lo + i]) : (T)~(T)0;
    __syncthreads();
    for (uint32_t k = 2; k <= P; k <<= 1) {
      for (uint32_t j = k >> 1; j > 0; j >>= 1) {
        // pair p: i = the p-th index with bit j clear, partner i + j
        for (uint32_t p = tid; p < (P >> 1); p += kSortThreads) {
          const uint32_t i = ((p & ~(j - 1)) << 1) | (p & (j - 1));
          const uint32_t l = i + j;
          const T x = buf[i], y = buf[l];
          const bool up = (i & k) == 0;
          if ((x > y) == up) { buf[i] = y; buf[l] = x; }
        }
        __syncthreads();
      }
    }
    for (uint32_t i = tid; i < n; i += kSortThreads) keys[q.lo + i] = buf[i];
    __syncthreads();
  }
}

struct QsLayout {
  QsSeg* lists[2];
  QsEq* eq;
  QsSeg* small;
  SegDesc* segs;
  uint64_t* splits;
  QsCounts* counts;
  void* batch;
  uint64_t maxseg;
  uint32_t slice;
  size_t bytes;
};

QsLayout qs_layout(void* base, uint64_t n) {
  QsLayout L{};
  L.maxseg = n / (kCut + 1) + 1;
  L.slice = (uint32_t)(L.maxseg < kSlice ? L.maxseg : kSlice);
  unsigned char* p = static_cast<unsigned char*>(base);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* r = p ? p + off : nullptr;
    off += (bytes + 255) / 256 * 256;
    return r;
  };
  L.lists[0] = reinterpret_cast<QsSeg*>(take(L.maxseg * sizeof(QsSeg)));
  L.lists[1] = reinterpret_cast<QsSeg*>(take(L.maxseg * sizeof(QsSeg)));
  L.eq = reinterpret_cast<QsEq*>(take(L.maxseg * sizeof(QsEq)));
  L.small = reinterpret_cast<QsSeg*>(take(2 * L.maxseg * sizeof(QsSeg)));
  L.segs = reinterpret_cast<SegDesc*>(take((size_t)L.slice * sizeof(SegDesc)));
  L.splits = reinterpret_cast<uint64_t*>(take((size_t)L.slice * 8));
  L.counts = reinterpret_cast<QsCounts*>(take(sizeof(QsCounts)));
  L.batch = take(batch_scratch_bytes(L.slice));
  L.bytes = off;
  return L;
}

cudaError_t read_counts(const QsLayout& L, QsCounts* host, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(host, L.counts, sizeof(QsCounts), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

}  // namespace

size_t quicksort_scratch_bytes(uint64_t n) { return qs_layout(nullptr, n).bytes; }

template <typename T>
cudaError_t launch_quicksort(T* keys, uint64_t n, uint64_t seed, void* scratch, void* host_words,
                             const BatchTuning& tune, uint32_t* bar, uint32_t* status,
                             LaunchCfg& cfg, const cudaEvent_t* ev, SortStats* stats) {
  cudaStream_t st = cfg.stream;
  *stats = SortStats{};
  if (n < 2) return cudaSuccess;
  const QsLayout L = qs_layout(scratch, n);
  const BatchScratch Bs = carve_batch_scratch(L.batch, L.slice, bar, status);
  QsCounts* hc = static_cast<QsCounts*>(host_words);
  cudaError_t e;
  uint64_t open = 0;
  uint32_t nsmall = 0, cur = 0, levels = 0;
  e = cudaMemsetAsync(L.counts, 0, sizeof(QsCounts), st);
  if (e != cudaSuccess) return e;
  {
    const QsSeg whole{0, n};
    // the whole array is the first open subarray, or the only small one
    e = cudaMemcpyAsync(n > kCut ? L.lists[0] : L.small, &whole, sizeof(QsSeg),
                        cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    if (n > kCut) open = 1; else nsmall = 1;
  }
  // optional timing: events around a stretch of launches, read after the
  // host's next synchronisation of the stream
  auto mark = [&](int k) -> cudaError_t { return ev ? cudaEventRecord(ev[k], st) : cudaSuccess; };
  auto elapsed = [&](float* acc) {
    float ms = 0.f;
    if (ev && cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess) *acc += ms;
  };
  auto sort_small = [&](uint32_t cnt) -> cudaError_t {
    if (cnt == 0) return cudaSuccess;
    const uint32_t grid = cnt < 8192 ? cnt : 8192;
    cudaError_t r = mark(0);
    if (r != cudaSuccess) return r;
    qs_small_sort_kernel<T><<<grid, kSortThreads, 0, st>>>(L.small, cnt, keys);
    cfg.launches++;
    if ((r = cudaGetLastError()) != cudaSuccess) return r;
    if (ev) {
      if ((r = mark(1)) != cudaSuccess || (r = cudaEventSynchronize(ev[1])) != cudaSuccess)
        return r;
      elapsed(&stats->sort_ms);
    }
    return cudaSuccess;
  };
  const unsigned long long* traffic = Bs.totals + 2;
  while (open > 0) {
    if (++levels > kMaxSortLevels) return cudaErrorUnknown;  // sizes shrink every level
    QsSeg* list = L.lists[cur];
    QsSeg* next = L.lists[cur ^ 1];
    e = cudaMemsetAsync(L.counts, 0, 16, st);  // the level's list sizes
    if (e == cudaSuccess) e = mark(0);
    if (e != cudaSuccess) return e;
    for (uint64_t o = 0; o < open; o += L.slice) {
      const uint32_t cnt = (uint32_t)(open - o < L.slice ? open - o : L.slice);
      const unsigned blocks = (cnt + 255) / 256;
      qs_build_kernel<T><<<blocks, 256, 0, st>>>(list + o, cnt, keys, seed + levels, L.segs);
      cfg.launches++;
      e = launch_batched<T>(L.segs, cnt, sm_stream(seed, levels), L.splits, Bs, tune, cfg);
      if (e != cudaSuccess) return e;
      qs_split_kernel<<<blocks, 256, 0, st>>>(list + o, cnt, L.segs, L.splits, next, L.small,
                                              L.eq, L.counts, traffic);
      cfg.launches++;
    }
    if ((e = mark(1)) != cudaSuccess) return e;
    if ((e = read_counts(L, hc, st)) != cudaSuccess) return e;
    elapsed(&stats->partition_ms);
    const uint32_t neq = hc->eq;
    if (neq > 0 && (e = mark(0)) != cudaSuccess) return e;
    for (uint32_t o = 0; o < neq; o += L.slice) {  // split off the keys equal to the pivot
      const uint32_t cnt = neq - o < L.slice ? neq - o : L.slice;
      const unsigned blocks = (cnt + 255) / 256;
      qs_build_eq_kernel<T><<<blocks, 256, 0, st>>>(L.eq + o, cnt, keys, L.segs);
      cfg.launches++;
      e = launch_batched<T>(L.segs, cnt, sm_stream(~seed, levels), L.splits, Bs, tune, cfg);
      if (e != cudaSuccess) return e;
      qs_split_eq_kernel<<<blocks, 256, 0, st>>>(L.eq + o, cnt, L.splits, next, L.small,
                                                 L.counts, traffic);
      cfg.launches++;
    }
    if (neq > 0) {
      if ((e = mark(1)) != cudaSuccess) return e;
      if ((e = read_counts(L, hc, st)) != cudaSuccess) return e;
      elapsed(&stats->partition_ms);
    }
    if ((e = sort_small(hc->small)) != cudaSuccess) return e;
    open = hc->next;
    cur ^= 1;
  }
  if ((e = sort_small(nsmall)) != cudaSuccess) return e;
  if ((e = read_counts(L, hc, st)) != cudaSuccess) return e;
  stats->levels = levels;
  stats->partition_keys = hc->part_keys;
  stats->sort_keys = hc->sort_keys + (n <= kCut ? n : 0);
  return cudaGetLastError();
}

template cudaError_t launch_quicksort<uint64_t>(uint64_t*, uint64_t, uint64_t, void*, void*,
                                                const BatchTuning&, uint32_t*, uint32_t*,
                                                LaunchCfg&, const cudaEvent_t*, SortStats*);
template cudaError_t launch_quicksort<uint32_t>(uint32_t*, uint64_t, uint64_t, void*, void*,
                                                const BatchTuning&, uint32_t*, uint32_t*,
                                                LaunchCfg&, const cudaEvent_t*, SortStats*);

}  // namespace lp
