// lp_batched.cu -- many independent partitions in one persistent cooperative
// launch.  Each segment is partitioned by the Recursive Smoothed Striding
// scheme of Sec. 4 (Partial Partition Steps on its open range [v_min, v_max))
// and finished on chip once its open range fits one CTA's shared memory.
//
// The kernel works in rounds, with grid barriers between phases:
//   plan  (CTA 0): for every open segment, the last step's v_min / v_max
//         become the new open range; a range one CTA can hold becomes a CTA
//         task, a larger one gets a step (line size b, g groups) from the
//         parameter rule; group counts are prefix-summed into a task list;
//   warp  every warp takes (segment, group) tasks from an atomic counter and
//         partitions that group (warp_pair_group, as in the single partition);
//         v_i go to the segment's record by atomic min / max;
//   cta   every CTA takes CTA tasks from an atomic counter: the open range is
//         partitioned in shared memory and the unaligned head and tail keys
//         of the segment are put in place; the split is written.
// The result of every segment is the partition the single-array entry points
// produce for it (same kernels per group, same on-chip finish); only the
// interleaving of work differs.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lp_batched.h"
#include "lp_coop.cuh"
#include "lp_launch.h"

namespace lp {

namespace {

enum : uint32_t { kSegOpen = 0, kSegCta = 1, kSegDone = 2 };

// Segment fields written by other CTAs are read through L2, never from L1.
__device__ __forceinline__ uint64_t L2(const uint64_t& x) {
  return __ldcg(reinterpret_cast<const unsigned long long*>(&x));
}
__device__ __forceinline__ unsigned long long L2(const unsigned long long& x) { return __ldcg(&x); }
__device__ __forceinline__ uint32_t L2(const uint32_t& x) {
  return __ldcg(reinterpret_cast<const unsigned int*>(&x));
}

template <typename T>
__device__ __forceinline__ T ldk(const T* p) {
  if constexpr (sizeof(T) == 8) return (T)__ldcg(reinterpret_cast<const unsigned long long*>(p));
  else return (T)__ldcg(reinterpret_cast<const unsigned int*>(p));
}

// Places the (< 16-byte) unaligned head [0, h) and tail [be, n) of a segment
// whose aligned body [h, be) is partitioned with body_count predecessors;
// returns the split.  One thread.
template <typename T>
__device__ uint64_t seg_fixup(T* keys, uint64_t n, uint64_t h, uint64_t be, uint64_t body_count,
                              T pivot) {
  const uint64_t m = h + body_count;
  uint64_t hp = 0, tp = 0;
  for (uint64_t p = 0; p < h; p++) hp += ldk(&keys[p]) <= pivot;
  for (uint64_t p = be; p < n; p++) tp += ldk(&keys[p]) <= pivot;
  const uint64_t t = body_count + hp + tp;
  uint64_t bad_s[16], bad_p[16];
  int ns = 0, np = 0;
  auto visit = [&](uint64_t p) {
    const bool pr = ldk(&keys[p]) <= pivot;
    if (p < t && !pr && ns < 16) bad_s[ns++] = p;
    if (p >= t && pr && np < 16) bad_p[np++] = p;
  };
  for (uint64_t p = 0; p < h; p++) visit(p);
  uint64_t r0 = m < t ? m : t, r1 = m < t ? t : m;
  if (r0 < h) r0 = h;
  if (r1 > be) r1 = be;
  for (uint64_t p = r0; p < r1; p++) visit(p);
  for (uint64_t p = be; p < n; p++) visit(p);
  const int q = ns < np ? ns : np;
  for (int j = 0; j < q; j++) {
    const T x = ldk(&keys[bad_s[j]]);
    keys[bad_s[j]] = ldk(&keys[bad_p[j]]);
    keys[bad_p[j]] = x;
  }
  return t;
}

template <typename T>
__global__ void __launch_bounds__(Tr<T, false>::Threads) batched_kernel(SegDesc* segs,
                                                                        uint32_t count,
                                                                        BatchArgs a,
                                                                        BatchScratch B) {
  using R = Tr<T, false>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ unsigned int flag;
  __shared__ uint32_t fetch;
  __shared__ unsigned long long tot_s[2];
  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;
  WarpSmem<T, false>& ws = reinterpret_cast<WarpSmem<T, false>*>(smem_raw)[warp];
  uint32_t phase = 0;
  const uint64_t total_warps = (uint64_t)gridDim.x * R::Warps;
  const uint32_t cta_cap = Coop<T, false>::Keys;
  TaskScratch S;
  S.status = B.status;
  S.bar = B.bar;

  // one round more than levels: the last forced step still gets its final plan
  for (uint32_t round = 0; round <= a.max_rounds; round++) {
    // ------------------------------------------------------------ plan
    if (blockIdx.x == 0) {
      unsigned long long wrun = 0, crun = 0;  // running totals of earlier chunks
      for (uint32_t c0 = 0; c0 < count; c0 += R::Threads) {
        const uint32_t s = c0 + tid;
        uint32_t gw = 0, gc = 0;
        if (s < count) {
          SegDesc& d = segs[s];
          const uint32_t level = L2(d.level);
          if (L2(d.state) == kSegOpen) {
            const uint64_t h = L2(d.h), be = L2(d.be);
            uint64_t lo = L2(d.lo), hi = L2(d.hi);
            if (level > 0) {  // the step of the last round left [vmin, vmax)
              lo = L2(d.vmin);
              hi = L2(d.vmax);
              if (level == 1) d.body_count = L2(d.count);
              if (lo < hi) {  // to the 16-byte grid of the body
                lo = h + ((lo - h) / R::A) * R::A;
                const uint64_t h2 = h + ((hi - h + R::A - 1) / R::A) * R::A;
                hi = h2 < be ? h2 : be;
              }
            }
            d.lo = lo;
            d.hi = hi;
            const uint64_t m = hi > lo ? hi - lo : 0;
            const uint64_t n = L2(d.n);
            if (m == 0 && level > 0) {
              const unsigned long long t = seg_fixup<T>(
                  reinterpret_cast<T*>(d.keys), n, h, be, L2(d.body_count), (T)L2(d.pivot));
              d.t = t;
              a.splits[s] = t;
              d.state = kSegDone;
            } else if ((level == 0 && n <= cta_cap) || (level > 0 && m <= cta_cap)) {
              d.state = kSegCta;
              gc = 1;
              atomicAdd(&B.totals[2], (unsigned long long)(level == 0 ? n : m));
            } else {
              atomicAdd(&B.totals[2], (unsigned long long)m);
              const StepParams P =
                  choose_params(m, R::K, a.group_workers, a.line_bytes, a.min_chunks);
              d.b = P.b;
              d.g = (level + 1 >= a.max_rounds) ? 1 : P.g;
              d.vmin = ~0ull;
              d.vmax = 0ull;
              d.count = 0ull;
              gw = (uint32_t)d.g;
            }
          }
        }
        // CTA-wide exclusive scans of gw and gc
        uint32_t iw = gw, ic = gc;
#pragma unroll
        for (uint32_t o = 1; o < 32; o <<= 1) {
          const uint32_t x = __shfl_up_sync(0xffffffffu, iw, o);
          const uint32_t y = __shfl_up_sync(0xffffffffu, ic, o);
          if (lane >= o) { iw += x; ic += y; }
        }
        uint32_t* wsw = reinterpret_cast<uint32_t*>(smem_raw);  // plan scratch (CTA 0)
        if (lane == 31) { wsw[warp] = iw; wsw[32 + warp] = ic; }
        __syncthreads();
        uint32_t bw = 0, bc = 0, tw = 0, tc = 0;
        for (uint32_t w = 0; w < R::Warps; w++) {
          const uint32_t x = wsw[w], y = wsw[32 + w];
          if (w < warp) { bw += x; bc += y; }
          tw += x;
          tc += y;
        }
        if (s < count) {
          B.wprefix[s] = wrun + bw + iw - gw;
          if (gc) B.ctalist[crun + bc + ic - gc] = s;
        }
        wrun += tw;
        crun += tc;
        __syncthreads();
      }
      if (tid == 0) {
        B.wprefix[count] = wrun;
        B.totals[0] = wrun;
        B.totals[1] = crun;
        B.counters[0] = 0u;
        B.counters[1] = 0u;
        __threadfence();
      }
    }
    if (!grid_barrier(S.bar, gridDim.x, &flag)) { if (tid == 0) atomicOr(S.status, kStatTimeout); return; }
    if (tid == 0) {
      tot_s[0] = __ldcg(&B.totals[0]);
      tot_s[1] = __ldcg(&B.totals[1]);
    }
    __syncthreads();
    const uint64_t W = tot_s[0], Cn = tot_s[1];
    if (W == 0 && Cn == 0) break;  // every segment is done

    // ------------------------------------------------------------ warp tasks
    if (W > 0) {
      if (lane == 0) {
        for (uint32_t st = 0; st < kStages; st++) mbar_init(&ws.bar[st], 1);
        fence_mbar_init();
        fence_proxy_async_smem();
      }
      __syncwarp();
      phase = 0;
      for (;;) {
        uint32_t k = 0;
        if (lane == 0) k = atomicAdd(&B.counters[0], 1u);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= W) break;
        // segment of task k: the last s with wprefix[s] <= k
        uint32_t lo_s = 0, hi_s = count;
        while (hi_s - lo_s > 1) {
          const uint32_t mid = (lo_s + hi_s) >> 1;
          if (__ldcg(&B.wprefix[mid]) <= k) lo_s = mid; else hi_s = mid;
        }
        const uint32_t s = lo_s;
        SegDesc& d = segs[s];
        const uint64_t i = k - __ldcg(&B.wprefix[s]);
        const uint64_t lo = L2(d.lo), hi = L2(d.hi);
        const uint64_t b = L2(d.b), g = L2(d.g);
        const uint32_t lev = L2(d.level);
        const StepGeom G = make_geom(hi - lo, b, g, level_seed(L2(d.seed), lev), 0);
        T* base = reinterpret_cast<T*>(d.keys) + lo;
        const int32_t nl = (int32_t)group_num_lines(G, i);
        uint64_t kk = 0;
        if (!warp_pair_group<T, false>(base, nullptr, G, (uint32_t)i, nl, (T)L2(d.pivot), ws,
                                       phase, kk, S.status))
          break;
        if (nl > 0 && lane == 0) {
          const unsigned long long v = lo + group_split_pos(G, i, (uint64_t)nl, kk);
          atomicMin(&d.vmin, v);
          atomicMax(&d.vmax, v);
          atomicAdd(&d.count, (unsigned long long)kk);
        }
      }
      __syncwarp();
      if (lane == 0)  // the CTA tasks reuse this shared memory
        for (uint32_t st = 0; st < kStages; st++) mbar_inval(&ws.bar[st]);
    }
    if (!grid_barrier(S.bar, gridDim.x, &flag)) { if (tid == 0) atomicOr(S.status, kStatTimeout); return; }

    // ------------------------------------------------------------ CTA tasks
    for (;;) {
      if (tid == 0) fetch = atomicAdd(&B.counters[1], 1u);
      __syncthreads();
      const uint32_t c = fetch;
      __syncthreads();
      if (c >= Cn) break;
      const uint32_t s = __ldcg(&B.ctalist[c]);
      SegDesc& d = segs[s];
      T* keys = reinterpret_cast<T*>(d.keys);
      const T pivot = (T)L2(d.pivot);
      if (L2(d.level) == 0) {  // the whole segment, any alignment
        const uint32_t cnt = cta_partition_smem<T, false>(keys, nullptr, (uint32_t)L2(d.n),
                                                          pivot, smem_raw);
        if (tid == 0) { d.t = cnt; a.splits[s] = cnt; d.state = kSegDone; }
      } else {  // the open range of the body, then the head and tail
        const uint64_t lo = L2(d.lo), hi = L2(d.hi);
        cta_partition_smem<T, false>(keys + lo, nullptr, (uint32_t)(hi - lo), pivot, smem_raw);
        if (tid == 0) {
          __threadfence_block();
          const unsigned long long t =
              seg_fixup<T>(keys, L2(d.n), L2(d.h), L2(d.be), L2(d.body_count), pivot);
          d.t = t;
          a.splits[s] = t;
          d.state = kSegDone;
        }
      }
      __syncthreads();
    }
    // segments that took a step move to the next level
    if (blockIdx.x == 0) {
      for (uint32_t s = tid; s < count; s += R::Threads)
        if (L2(segs[s].state) == kSegOpen) segs[s].level = L2(segs[s].level) + 1;
    }
    if (!grid_barrier(S.bar, gridDim.x, &flag)) { if (tid == 0) atomicOr(S.status, kStatTimeout); return; }
  }
}

// Per-segment set-up on the device: the 16-byte aligned body of each segment.
template <typename T>
__global__ void batch_setup_kernel(SegDesc* segs, uint32_t count, uint64_t seed,
                                   unsigned long long* traffic) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s == 0) *traffic = 0ull;
  if (s >= count) return;
  SegDesc& d = segs[s];
  constexpr uint32_t K = sizeof(T), A = 16 / sizeof(T);
  const uintptr_t addr = reinterpret_cast<uintptr_t>(d.keys);
  uint64_t h = ((16 - (addr & 15)) & 15) / K;
  if (h > d.n) h = d.n;
  d.h = h;
  d.be = h + ((d.n - h) / A) * A;
  d.lo = h;
  d.hi = d.be;
  d.level = 0;
  d.state = kSegOpen;
  // the offsets X of a segment depend on the batch seed and the segment's
  // salt only, not on its place in the list
  d.seed = sm_stream(seed, d.salt);
  d.vmin = ~0ull;
  d.vmax = 0ull;
  d.count = 0ull;
  d.body_count = 0ull;
  d.t = 0ull;
}

}  // namespace

size_t batch_scratch_bytes(uint32_t count) {
  return (((size_t)count + 1) * 8 + 255) / 256 * 256 + ((size_t)count * 4 + 255) / 256 * 256 + 256;
}

BatchScratch carve_batch_scratch(void* base, uint32_t count, uint32_t* bar, uint32_t* status) {
  unsigned char* p = static_cast<unsigned char*>(base);
  BatchScratch B;
  B.wprefix = reinterpret_cast<unsigned long long*>(p);
  p += (((size_t)count + 1) * 8 + 255) / 256 * 256;
  B.ctalist = reinterpret_cast<uint32_t*>(p);
  p += ((size_t)count * 4 + 255) / 256 * 256;
  B.totals = reinterpret_cast<unsigned long long*>(p);
  B.counters = reinterpret_cast<uint32_t*>(p + 64);
  B.bar = bar;
  B.status = status;
  return B;
}

template <typename T>
cudaError_t launch_batched(SegDesc* d_segs, uint32_t count, uint64_t seed, uint64_t* d_splits,
                           const BatchScratch& Bs, const BatchTuning& tune, LaunchCfg& cfg) {
  using R = Tr<T, false>;
  cudaStream_t st = cfg.stream;
  if (count == 0) return cudaSuccess;
  batch_setup_kernel<T><<<(count + 255) / 256, 256, 0, st>>>(d_segs, count, seed,
                                                              Bs.totals + 2);
  cfg.launches++;
  cudaError_t e = cudaMemsetAsync(Bs.bar, 0, 8, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(Bs.status, 0, 4, st);
  if (e != cudaSuccess) return e;
  BatchArgs a;
  a.splits = d_splits;
  a.max_rounds = kMaxLevels;
  uint32_t grid = cfg.grid;
  if (tune.ctas && tune.ctas < grid) grid = tune.ctas;
  a.group_workers = tune.group_workers ? tune.group_workers : (uint64_t)grid * R::Warps;
  a.line_bytes = tune.line_bytes ? tune.line_bytes : R::LineBytes;
  a.min_chunks = tune.min_chunks ? tune.min_chunks : 64;
  const size_t smem = level_smem_bytes<T, false>();  // attribute set by batched_prepare
  e = launch_cooperative(batched_kernel<T>, grid, R::Threads, smem, st, d_segs, count, a, Bs);
  cfg.launches++;
  return e;
}

template <typename T>
cudaError_t batched_prepare(int device, uint32_t* grid) {
  using R = Tr<T, false>;
  const size_t smem = level_smem_bytes<T, false>();
  cudaError_t e = cudaFuncSetAttribute(batched_kernel<T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int sms = 0, per = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batched_kernel<T>, R::Threads, smem);
  if (e != cudaSuccess) return e;
  if (per < 1) return cudaErrorInvalidConfiguration;
  *grid = (uint32_t)(sms * per);  // every CTA resident: the grid barrier needs it
  return cudaSuccess;
}
template cudaError_t batched_prepare<uint64_t>(int, uint32_t*);
template cudaError_t batched_prepare<uint32_t>(int, uint32_t*);

template cudaError_t launch_batched<uint64_t>(SegDesc*, uint32_t, uint64_t, uint64_t*,
                                              const BatchScratch&, const BatchTuning&,
                                              LaunchCfg&);
template cudaError_t launch_batched<uint32_t>(SegDesc*, uint32_t, uint64_t, uint64_t*,
                                              const BatchScratch&, const BatchTuning&,
                                              LaunchCfg&);

}  // namespace lp
