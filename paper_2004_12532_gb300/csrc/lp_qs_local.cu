// lp_qs_local.cu -- the tail of the quicksort on the partition (Sec. 5, "A
// Full Quicksort": the top levels partition in parallel, each subproblem then
// on its own).  Once the level-synchronous levels have few subarrays left,
// each of them is sorted by one CTA, depth first, from a stack in shared
// memory:
//   at most kQsCut keys   the shared-memory sort (cta_sort_small);
//   larger                partitioned by [x <= p], p the median of seeded keys
//                         (qs_item_hash, as in the levels): the 16-byte
//                         aligned body by one on-chip partition once one
//                         CTA's shared memory holds the open range
//                         (cta_partition_bulk), before that by Partial
//                         Partition Steps (Sec. 4) whose groups the CTA's
//                         warps take from a counter; the head and tail by
//                         seg_fixup; the two children are pushed, the larger
//                         first, so the smaller is taken next and the stack
//                         stays shallow;
//   equal keys            as in the levels: a subarray with no key above
//                         p > 0 is partitioned again by [x < p], and the keys
//                         equal to p are final.
// CTAs take subarrays from a counter and never wait for one another (no
// grid-wide barrier; a normal launch): memory-bound partitions and
// compute-bound sorts of different CTAs overlap, and a subarray's later
// levels find its keys in L2.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lp_fixup.cuh"
#include "lp_qs.cuh"
#include "lp_qs_pivot.cuh"
#include "lp_qs_sort.cuh"
#include "lp_smoothed.cuh"

namespace lp {

namespace {

constexpr uint32_t kLocalStack = 64;  // pieces on a CTA's stack, at most (depth <= ~20)
constexpr int kLocalMaxSteps = 6;     // steps on one piece before a one-group step ends it

struct LocalItem {
  uint64_t lo, n;
  uint64_t pivot;  // of an equal-key piece: partitioned by [x <= pivot - 1]
  uint32_t level, eq;
};

template <typename T>
__global__ void __launch_bounds__(Tr<T, false>::Threads, 2)
    qs_local_kernel(T* keys, const QsItem* list, uint32_t count, uint32_t level,
                    uint64_t seed, uint32_t samples, unsigned long long* fetch,
                    unsigned long long* acc, uint32_t* status) {
  using R = Tr<T, false>;
  static_assert(R::Threads == kQsSortThreads, "the steps and the sort share the CTA");
  constexpr uint32_t FULL = 0xffffffffu;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ LocalItem stack[kLocalStack];
  __shared__ LocalItem cur;
  __shared__ uint32_t depth, abort_flag, next_group, have;
  __shared__ unsigned long long s_vmin, s_vmax, s_count;
  __shared__ T s_pivot;
  __shared__ __align__(8) uint64_t cta_bar;  // the on-chip partitions' bulk copies
  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;
  WarpSmem<T, false>& ws = reinterpret_cast<WarpSmem<T, false>*>(smem_raw)[warp];
  uint32_t phase = 0, cta_parity = 0;
  bool warp_mode = false;  // the warps' stage barriers are initialised
  unsigned long long streamed = 0, sorted_keys = 0;  // thread 0's tallies
  unsigned long long ns_sort = 0, ns_part = 0;       // ... and its time in each kind
  if (tid == 0) {
    mbar_init(&cta_bar, 1);
    fence_mbar_init();
    abort_flag = 0u;
    depth = 0u;
  }
  __syncthreads();

  // The dynamic shared memory serves either the warps' line stages (steps) or
  // one whole-CTA buffer (on-chip partition, sort); the stage barriers live in
  // it, so they are invalidated before the memory is reused and set up again
  // after.  Every thread calls these (CTA-uniform control).
  auto to_cta_mode = [&]() {
    __syncthreads();
    if (warp_mode) {
      if (lane == 0)
        for (uint32_t s = 0; s < R::Stages; s++) mbar_inval(&ws.bar[s]);
      warp_mode = false;
      __syncthreads();
    }
  };
  auto to_warp_mode = [&]() {
    __syncthreads();
    if (!warp_mode) {
      if (lane == 0) {
        for (uint32_t s = 0; s < R::Stages; s++) mbar_init(&ws.bar[s], 1);
        fence_mbar_init();
        fence_proxy_async_smem();
      }
      phase = 0;
      warp_mode = true;
      __syncthreads();
    }
  };

  for (;;) {
    // the next subarray of the list
    if (tid == 0) {
      have = 0u;
      if (!abort_flag) {
        const unsigned long long r = atomicAdd(fetch, 1ull);
        if (r < count) {
          const QsItem q = list[r];
          stack[0] = LocalItem{q.lo, q.n, q.pivot, level, (uint32_t)q.eq};
          depth = 1u;
          have = 1u;
        }
      }
    }
    __syncthreads();
    if (!have) break;
    for (;;) {
      // this CTA's writes to the keys are ordered before the bulk copies
      // (async proxy) that may read them for the next piece
      fence_proxy_async_global();
      __syncthreads();
      if (tid == 0) {
        have = 0u;
        if (depth > 0 && !abort_flag) {
          cur = stack[--depth];
          have = 1u;
        }
      }
      __syncthreads();
      if (!have) break;
      const LocalItem it = cur;
      if (it.n <= 1) continue;
      const uint64_t t_piece = tid == 0 ? global_timer_ns() : 0;
      if (it.n <= kQsCut && !it.eq) {
        to_cta_mode();
        cta_sort_small<T>(keys + it.lo, (uint32_t)it.n, smem_raw);
        if (tid == 0) {
          sorted_keys += it.n;
          ns_sort += global_timer_ns() - t_piece;
        }
        continue;
      }
      const uint64_t hsh = qs_item_hash(seed, it.level, it.lo, it.n);
      if (tid == 0) {
        if (it.eq) s_pivot = (T)(it.pivot - 1);
        else if (samples == kQsSamplesMax) s_pivot = qs_median<kQsSamplesMax>(keys, it.lo, it.n, hsh);
        else s_pivot = qs_median<3>(keys, it.lo, it.n, hsh);
      }
      __syncthreads();
      const T p = s_pivot;
      T* const base = keys + it.lo;
      const uint64_t n = it.n;
      const uintptr_t addr = reinterpret_cast<uintptr_t>(base);
      uint64_t h = ((16 - (addr & 15)) & 15) / R::K;
      if (h > n) h = n;
      const uint64_t be = h + ((n - h) / R::A) * R::A;  // the aligned body [h, be)
      uint64_t rlo = h, rhi = be, body_count = 0;
      bool first = true;
      for (int step = 0; rhi > rlo; step++) {
        const uint64_t m = rhi - rlo;
        if (m <= CtaBulk<T>::Keys) {  // the open range fits on chip
          to_cta_mode();
          const uint32_t c = cta_partition_bulk<T>(base + rlo, (uint32_t)m, p, smem_raw,
                                                   &cta_bar, cta_parity, status);
          if (c == ~0u) {
            if (tid == 0) abort_flag = 1u;
          } else if (first) {
            body_count = c;
          }
          if (tid == 0) streamed += m;
          break;
        }
        to_warp_mode();
        StepParams P = choose_params(m, R::K, R::Warps, R::LineBytes);
        if (step >= kLocalMaxSteps) P.g = 1;  // one warp partitions what is left
        const StepGeom G = make_geom(m, P.b, P.g, level_seed(hsh, (uint64_t)step + 1), 0);
        if (tid == 0) {
          s_vmin = ~0ull;
          s_vmax = 0ull;
          s_count = 0ull;
          next_group = 0u;
        }
        __syncthreads();
        for (;;) {
          uint32_t i = 0;
          if (lane == 0) i = atomicAdd(&next_group, 1u);
          i = __shfl_sync(FULL, i, 0);
          if (i >= G.g) break;
          const int32_t nl = (int32_t)group_num_lines(G, i);
          uint64_t k = 0;
          if (!warp_pair_group<T, false>(base + rlo, nullptr, G, i, nl, p, ws, phase, k,
                                         status)) {
            if (lane == 0) atomicExch(&abort_flag, 1u);
            break;
          }
          if (nl > 0 && lane == 0) {
            const unsigned long long v = rlo + group_split_pos(G, i, (uint64_t)nl, k);
            atomicMin(&s_vmin, v);
            atomicMax(&s_vmax, v);
            atomicAdd(&s_count, (unsigned long long)k);
          }
        }
        fence_proxy_async_global();  // the step's writes before the next step's copies
        __syncthreads();
        if (abort_flag) break;
        if (first) body_count = s_count;  // the first step counts the whole body
        first = false;
        if (tid == 0) streamed += m;
        uint64_t lo2 = s_vmin, hi2 = s_vmax;
        if (lo2 >= hi2) break;  // partitioned
        lo2 = h + ((lo2 - h) / R::A) * R::A;  // to the 16-byte grid of the body
        hi2 = h + ((hi2 - h + R::A - 1) / R::A) * R::A;
        rlo = lo2;
        rhi = hi2 < be ? hi2 : be;
      }
      __syncthreads();
      if (abort_flag) break;
      if (tid == 0) {
        const uint64_t t = seg_fixup<T>(base, n, h, be, body_count, p);
        auto push = [&](uint64_t lo, uint64_t m, uint64_t pv, uint32_t eq) {
          if (m <= 1) return;
          if (depth < kLocalStack) {
            stack[depth++] = LocalItem{lo, m, pv, it.level + 1, eq};
          } else {  // never expected: the smaller child is always taken first
            atomicOr(status, kStatRing);
            abort_flag = 1u;
          }
        };
        if (it.eq) {
          push(it.lo, t, 0ull, 0u);  // below p; the rest equals p and is final
        } else if (t == n) {
          if (p != 0) push(it.lo, n, (uint64_t)p, 1u);  // no key above p: split off == p
        } else if (t >= n - t) {
          push(it.lo, t, 0ull, 0u);
          push(it.lo + t, n - t, 0ull, 0u);
        } else {
          push(it.lo + t, n - t, 0ull, 0u);
          push(it.lo, t, 0ull, 0u);
        }
        ns_part += global_timer_ns() - t_piece;
      }
    }
    __syncthreads();
    if (abort_flag) break;
  }
  if (tid == 0) {
    atomicAdd(&acc[0], streamed);
    atomicAdd(&acc[1], sorted_keys);
    atomicAdd(&acc[3], ns_sort);
    atomicAdd(&acc[4], ns_part);
  }
}

}  // namespace

template <typename T>
cudaError_t qs_local_grid(int device, uint32_t* grid) {
  using R = Tr<T, false>;
  const size_t smem = level_smem_bytes<T, false>();
  cudaError_t e = cudaFuncSetAttribute(qs_local_kernel<T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int sms = 0, per = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, qs_local_kernel<T>, R::Threads, smem);
  if (e != cudaSuccess) return e;
  *grid = (uint32_t)(sms * (per < 1 ? 1 : per));
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_qs_local(T* keys, const QsItem* list, uint32_t count, uint32_t level,
                            uint64_t seed, uint32_t samples, unsigned long long* acc,
                            uint32_t* status, uint32_t grid, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  unsigned long long* fetch = acc + 2;
  cudaError_t e = cudaMemsetAsync(fetch, 0, 8, st);
  if (e != cudaSuccess) return e;
  const uint32_t g = count < grid ? count : grid;
  qs_local_kernel<T><<<g, Tr<T, false>::Threads, level_smem_bytes<T, false>(), st>>>(
      keys, list, count, level, seed, samples, fetch, acc, status);
  return cudaGetLastError();
}

template cudaError_t qs_local_grid<uint64_t>(int, uint32_t*);
template cudaError_t qs_local_grid<uint32_t>(int, uint32_t*);
template cudaError_t launch_qs_local<uint64_t>(uint64_t*, const QsItem*, uint32_t, uint32_t,
                                               uint64_t, uint32_t, unsigned long long*,
                                               uint32_t*, uint32_t, cudaStream_t);
template cudaError_t launch_qs_local<uint32_t>(uint32_t*, const QsItem*, uint32_t, uint32_t,
                                               uint64_t, uint32_t, unsigned long long*,
                                               uint32_t*, uint32_t, cudaStream_t);

}  // namespace lp
