// lp_kernels.cu -- kernels of the Recursive Smoothed Striding partition
// (Sec. 4 of arXiv 2004.12532) and their host launchers.
//
//   desc_init_kernel   resets the level descriptors, status and grid barrier
//   partition_kernel   the whole recursion in one cooperative launch: level 0
//                      on the caller's range, then each level on the range
//                      [v_min, v_max) the previous one left open (Sec. 4,
//                      "Recurse on A[v_min] .. A[v_max - 1]"), a grid barrier
//                      between levels; once the open range fits in the CTAs'
//                      shared memory, the base case partitions it on chip
//   level_kernel       one Partial Partition Step with explicit parameters
//                      (the lp_smoothed_step entry point)
//   finalize_kernel    places the (< 16-byte) unaligned head and tail keys and
//                      writes the split t
//   fill kernels       seeded synthetic inputs (SplitMix64), harness only
#include <cuda_runtime.h>
#include <stdint.h>

#include "lp_coop.cuh"
#include "lp_launch.h"
#include "lp_smoothed.cuh"

namespace lp {

size_t level_desc_bytes() { return sizeof(LevelDesc); }

namespace {
// groups per warp at level 0 of the recursive partition, at most (measured:
// 8 for keys, 16 for key + payload pairs at 2^30 keys on GB300)
template <bool KV>
constexpr uint64_t kLevel0GroupsPerWarp = KV ? 16 : 8;
// ... and chunks per group, at least (shorter groups cost more than they save)
constexpr uint32_t kLevel0MinChunks = 128;
}  // namespace

// ------------------------------------------------------------ scratch layout
size_t task_scratch_bytes(uint32_t grid) {
  return sizeof(LevelDesc) * (kMaxLevels + 1) /* levels, handoff */ + 64 /* status */ +
         64 /* barrier, t_end */ + ((size_t)grid * 4 + 63) / 64 * 64 /* counts */;
}

TaskScratch carve_scratch(void* base, uint32_t grid) {
  (void)grid;
  unsigned char* p = static_cast<unsigned char*>(base);
  TaskScratch S;
  S.desc = reinterpret_cast<LevelDesc*>(p);
  p += sizeof(LevelDesc) * kMaxLevels;
  S.handoff = reinterpret_cast<LevelDesc*>(p);
  p += sizeof(LevelDesc);
  S.status = reinterpret_cast<uint32_t*>(p);
  S.split = reinterpret_cast<uint64_t*>(p + 8);
  p += 64;
  S.bar = reinterpret_cast<uint32_t*>(p);
  S.t_end = reinterpret_cast<unsigned long long*>(p + 8);
  static_assert(16 + 4 * kMaxLevels <= 64, "the group counters share the barrier's 64 bytes");
  S.fetch = reinterpret_cast<uint32_t*>(p + 16);
  p += 64;
  S.counts = reinterpret_cast<uint32_t*>(p);
  return S;
}

__global__ void desc_init_kernel(TaskScratch S) {
  const int t = threadIdx.x;
  if (t <= kMaxLevels) {  // the levels, then the handoff record (empty)
    LevelDesc& d = t < kMaxLevels ? S.desc[t] : *S.handoff;
    d.vmin = ~0ull;
    d.vmax = 0ull;
    d.count = 0ull;
    d.lo = d.hi = d.b = d.g = d.t_start = 0ull;
    if (t < kMaxLevels) S.fetch[t] = 0u;
  }
  if (t == 0) {
    *S.status = 0u;
    S.bar[0] = 0u;
    S.bar[1] = 0u;
    *S.t_end = 0ull;
  }
}

// Extends [lo, hi) outward to 16-byte boundaries of the body [body_lo,
// body_hi): keys added on the left are predecessors already in final place and
// keys added on the right successors, so partitioning the wider range is
// equivalent.
__device__ __forceinline__ void align_range(uint64_t body_lo, uint64_t body_hi, uint32_t A,
                                            uint64_t& lo, uint64_t& hi) {
  lo = body_lo + ((lo - body_lo) / A) * A;
  const uint64_t h2 = body_lo + ((hi - body_lo + A - 1) / A) * A;
  hi = h2 < body_hi ? h2 : body_hi;
}

struct PartArgs {
  uint64_t body_lo, body_hi;  // 16-byte aligned body of the array
  uint64_t pivot, seed;
  int strided;                // level 0 with X == 0 (the Strided Algorithm)
  int max_levels;             // 1: level 0 only, the open range left for a cleanup
  int handoff;                // 1: a range the recursion cannot finish goes to S.handoff
  int level_cap;              // with handoff: the level at which an open range is handed over
};

// The whole recursion in one cooperative launch; see the file comment.
template <typename T, bool KV>
__global__ void __launch_bounds__(Tr<T, KV>::Threads, 2) partition_kernel(T* keys, uint64_t* vals,
                                                                       PartArgs a,
                                                                       TaskScratch S) {
  using R = Tr<T, KV>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ unsigned int bar_flag;
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  WarpSmem<T, KV>& ws = reinterpret_cast<WarpSmem<T, KV>*>(smem_raw)[warp];
  if (lane == 0) {
    for (uint32_t s = 0; s < Tr<T, KV>::Stages; s++) mbar_init(&ws.bar[s], 1);
    fence_mbar_init();
    fence_proxy_async_smem();
  }
  __syncwarp();
  uint32_t phase = 0;
  const uint64_t total_warps = (uint64_t)gridDim.x * R::Warps;
  const uint64_t coop_cap = (uint64_t)gridDim.x * Coop<T, KV>::Keys;
  const T pivot = (T)a.pivot;
  uint64_t prev_n = 0;  // the range of the level before
  int stalls = 0;       // levels that left at least 7/8 of the range before them open

  for (int L = 0; L < a.max_levels; L++) {
    uint64_t lo, hi;
    if (L == 0) {
      lo = a.body_lo;
      hi = a.body_hi;
    } else {
      lo = __ldcg(&S.desc[L - 1].vmin);
      hi = __ldcg(&S.desc[L - 1].vmax);
    }
    if (lo >= hi) break;
    align_range(a.body_lo, a.body_hi, R::A, lo, hi);
    const uint64_t n = hi - lo;
    if (leader) {
      S.desc[L].lo = lo;
      S.desc[L].hi = hi;
      S.desc[L].t_start = global_timer_ns();
    }
    T* base = keys + lo;
    uint64_t* vbase = KV ? vals + lo : nullptr;

    if (n <= coop_cap) {  // the paper's base case, on chip
      if (lane == 0)  // the finish reuses the stages' shared memory
        for (uint32_t s2 = 0; s2 < Tr<T, KV>::Stages; s2++) mbar_inval(&ws.bar[s2]);
      __syncthreads();
      const uint64_t t = coop_finish<T, KV>(base, vbase, n, pivot, S, smem_raw, &bar_flag);
      if (t == ~0ull) {
        if (threadIdx.x == 0) atomicOr(S.status, kStatTimeout | kSitePartition);
      } else if (leader) {
        S.desc[L].vmin = lo + t;
        S.desc[L].vmax = lo + t;
        S.desc[L].count = t;
        S.desc[L].b = 0;
        S.desc[L].g = 0;
      }
      break;
    }

    // residual-shrink guard: the open range goes to the low-space partition
    // (launched after this kernel) at the level cap, or once kShrinkTries
    // levels, each with fresh offsets X, have failed to shrink it by 1/8;
    // every CTA sees the same ranges, so all take the same branch
    if (a.handoff && L > 0) {
      if (n >= prev_n - prev_n / 8) stalls++;
      if (L >= a.level_cap || stalls >= kShrinkTries) {
        if (leader) {
          S.handoff->vmin = lo;
          S.handoff->vmax = hi;
          S.desc[L].b = 0;
          S.desc[L].g = ~0ull;  // marks the handoff in the level records
        }
        break;
      }
    }
    prev_n = n;

    // a Partial Partition Step (parameter rule of lp_plan.h); without a
    // handoff the last level, should a range still be open, is one group.  Warps take groups one at a
    // time from a counter, so that they finish together.  Level 0 of the
    // recursion has up to kLevel0GroupsPerWarp groups per warp (the tail of a
    // level costs more than the wider open range more groups leave); later
    // levels, and a single step whose open range another algorithm cleans
    // up, one per warp (longer groups leave a narrower open range)
    const bool wide = L == 0 && a.max_levels > 1;
    const uint64_t workers = wide ? total_warps * kLevel0GroupsPerWarp<KV> : total_warps;
    const StepParams P =
        wide ? choose_params(n, R::K, workers, R::LineBytes, kLevel0MinChunks)
             : choose_params(n, R::K, workers, R::LineBytes);
    const uint64_t b = P.b;
    const uint64_t g = (!a.handoff && L == kMaxLevels - 1) ? 1 : P.g;
    if (leader) { S.desc[L].b = b; S.desc[L].g = g; }
    const StepGeom G = make_geom(n, b, g, level_seed(a.seed, (uint64_t)L),
                                 (a.strided && L == 0) ? 1 : 0);
    for (;;) {
      uint32_t i = 0;
      if (lane == 0) i = atomicAdd(&S.fetch[L], 1u);
      i = __shfl_sync(0xffffffffu, i, 0);
      if (i >= G.g) break;
      const int32_t nl = (int32_t)group_num_lines(G, i);
      uint64_t k = 0;
      if (!warp_pair_group<T, KV>(base, vbase, G, (uint32_t)i, nl, pivot, ws, phase, k,
                                  S.status))
        break;  // the status is set; the barrier below still runs
      if (nl > 0 && lane == 0) {
        const unsigned long long v = lo + group_split_pos(G, i, (uint64_t)nl, k);
        atomicMin(&S.desc[L].vmin, v);
        atomicMax(&S.desc[L].vmax, v);
        atomicAdd(&S.desc[L].count, (unsigned long long)k);
      }
    }
    // a one-group level is one warp's partition of the whole range
    if (!grid_barrier(S.bar, gridDim.x, &bar_flag,
                      g == 1 ? wait_limit_for_bytes(n * (R::K + (KV ? 8u : 0u)))
                             : kWaitLimitNs)) {
      if (threadIdx.x == 0) atomicOr(S.status, kStatTimeout | kSitePartition);
      break;
    }
    // stop on an error raised anywhere in this level; one thread reads the
    // status so that the whole CTA takes the same branch
    if (threadIdx.x == 0) bar_flag = __ldcg(S.status) == 0u ? 1u : 0u;
    __syncthreads();
    if (!bar_flag) break;
  }
  if (leader) *S.t_end = global_timer_ns();
}

// One Partial Partition Step with explicit parameters on [a.lo, a.hi).
template <typename T, bool KV>
__global__ void __launch_bounds__(Tr<T, KV>::Threads, 2) level_kernel(T* keys, uint64_t* vals,
                                                                   LevelArgs a, LevelDesc* out,
                                                                   uint32_t* status) {
  using R = Tr<T, KV>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const uint64_t lo = a.lo, n = a.hi - a.lo;
  const uint64_t total_warps = (uint64_t)gridDim.x * R::Warps;
  const StepGeom G = make_geom(n, a.fixed_b, a.fixed_g, level_seed(a.seed, a.level), a.strided);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    out->lo = lo; out->hi = a.hi; out->b = a.fixed_b; out->g = a.fixed_g;
  }
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const uint64_t gw = (uint64_t)blockIdx.x * R::Warps + warp;
  if (gw >= G.g) return;  // warps are independent: no CTA barrier below
  WarpSmem<T, KV>& ws = reinterpret_cast<WarpSmem<T, KV>*>(smem_raw)[warp];
  if (lane == 0) {
    for (uint32_t s = 0; s < Tr<T, KV>::Stages; s++) mbar_init(&ws.bar[s], 1);
    fence_mbar_init();
    fence_proxy_async_smem();
  }
  __syncwarp();
  uint32_t phase = 0;
  T* base = keys + lo;
  uint64_t* vbase = KV ? vals + lo : nullptr;
  const T pivot = (T)a.pivot;
  for (uint64_t i = gw; i < G.g; i += total_warps) {
    const int32_t nl = (int32_t)group_num_lines(G, i);
    uint64_t k = 0;
    if (!warp_pair_group<T, KV>(base, vbase, G, (uint32_t)i, nl, pivot, ws, phase, k, status))
      break;
    if (nl > 0 && lane == 0) {
      const unsigned long long v = lo + group_split_pos(G, i, (uint64_t)nl, k);
      atomicMin(&out->vmin, v);
      atomicMax(&out->vmax, v);
      atomicAdd(&out->count, (unsigned long long)k);
    }
  }
}

// Head keys [0, h) and tail keys [body_end, n) lie outside the 16-byte aligned
// body that the levels partitioned.  With the body split at m = h + count,
// every misplaced key is in the head, the tail, or the body between m and the
// final split t; there are at most a dozen, and one thread swaps them.  After
// a failure raised earlier (a wait that gave up) the body's count is partial:
// nothing is scanned or moved, and the split reads UINT64_MAX, never a valid
// split.
template <typename T, bool KV>
__global__ void finalize_kernel(T* keys, uint64_t* vals, uint64_t n, uint64_t h,
                                uint64_t body_end, T pivot, TaskScratch S) {
  if (threadIdx.x != 0) return;
  if (__ldcg(S.status) != 0u) {
    *S.split = ~0ull;
    return;
  }
  const uint64_t cb = S.desc[0].count;
  const uint64_t m = h + cb;
  uint64_t hp = 0, tp = 0;
  for (uint64_t p = 0; p < h; p++) hp += keys[p] <= pivot;
  for (uint64_t p = body_end; p < n; p++) tp += keys[p] <= pivot;
  const uint64_t t = cb + hp + tp;
  uint64_t bad_s[32], bad_p[32];
  int ns = 0, np = 0;
  auto visit = [&](uint64_t p) {
    const bool pr = keys[p] <= pivot;
    if (p < t && !pr && ns < 32) bad_s[ns++] = p;
    if (p >= t && pr && np < 32) bad_p[np++] = p;
  };
  for (uint64_t p = 0; p < h; p++) visit(p);
  uint64_t r0 = m < t ? m : t, r1 = m < t ? t : m;
  if (r0 < h) r0 = h;
  if (r1 > body_end) r1 = body_end;
  for (uint64_t p = r0; p < r1; p++) visit(p);
  for (uint64_t p = body_end; p < n; p++) visit(p);
  if (ns != np || ns >= 32) {
    atomicOr(S.status, kStatRing);
  } else {
    for (int q = 0; q < ns; q++) {
      T x = keys[bad_s[q]];
      keys[bad_s[q]] = keys[bad_p[q]];
      keys[bad_p[q]] = x;
      if constexpr (KV) {
        uint64_t y = vals[bad_s[q]];
        vals[bad_s[q]] = vals[bad_p[q]];
        vals[bad_p[q]] = y;
      }
    }
  }
  *S.split = t;
}

// Whole partition of an array of n <= small_limit keys in one CTA (any
// alignment), for arrays too short for a 16-byte aligned body.
uint64_t small_limit(uint32_t key_bytes, bool kv) {
  return kFinishBytes / (key_bytes + (kv ? 8u : 0u));
}

template <typename T, bool KV>
__global__ void __launch_bounds__(Tr<T, KV>::Threads) small_kernel(T* keys, uint64_t* vals,
                                                                   uint32_t n, T pivot,
                                                                   uint64_t* split) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const uint32_t cnt = cta_partition_smem<T, KV>(keys, vals, n, pivot, smem_raw);
  if (threadIdx.x == 0) *split = cnt;
}

template <typename T, bool KV>
static size_t stream_smem_bytes() {
  return level_smem_bytes<T, KV>();
}

template <typename T, bool KV>
cudaError_t streaming_grid(int device, uint32_t* grid) {
  cudaError_t e;
  const size_t smem = stream_smem_bytes<T, KV>();
  e = cudaFuncSetAttribute(partition_kernel<T, KV>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(level_kernel<T, KV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(small_kernel<T, KV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  if (e != cudaSuccess) return e;
  int sms = 0, per = 0, per2 = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, partition_kernel<T, KV>,
                                                    Tr<T, KV>::Threads, smem);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, level_kernel<T, KV>,
                                                    Tr<T, KV>::Threads, smem);
  if (e != cudaSuccess) return e;
  if (per2 < per) per = per2;
  if (per < 1) per = 1;
  *grid = (uint32_t)(sms * per);
  return cudaSuccess;
}

template <typename T, bool KV>
bool smoothed_may_hand_off(uint64_t n, uint32_t grid) {
  using R = Tr<T, KV>;
  // the body is at most n keys; the on-chip base case takes it whole at level 0
  return n > small_limit(R::K, KV) && n > (uint64_t)grid * Coop<T, KV>::Keys + 2 * R::A;
}

template <typename T, bool KV>
cudaError_t launch_smoothed(T* keys, uint64_t* vals, uint64_t n, T pivot, uint64_t seed,
                            int strided, const TaskScratch& S, LaunchCfg& cfg, void* handoff_var,
                            uint32_t level_cap) {
  using R = Tr<T, KV>;
  cudaStream_t st = cfg.stream;
  const size_t smem = stream_smem_bytes<T, KV>();
  desc_init_kernel<<<1, 32, 0, st>>>(S);
  cfg.launches++;
  if (n <= small_limit(R::K, KV)) {
    if (cfg.events) cudaEventRecord(cfg.events[0], st);
    small_kernel<T, KV><<<1, R::Threads, smem, st>>>(keys, vals, (uint32_t)n, pivot, S.split);
    cfg.launches++;
    if (cfg.events) cudaEventRecord(cfg.events[1], st);
    return cudaGetLastError();
  }
  const uintptr_t addr = reinterpret_cast<uintptr_t>(keys);
  const uint64_t h = ((16 - (addr & 15)) & 15) / R::K;
  const uint64_t body_end = h + ((n - h) / R::A) * R::A;
  PartArgs a;
  a.body_lo = h;
  a.body_hi = body_end;
  a.pivot = (uint64_t)pivot;
  a.seed = seed;
  a.strided = strided;
  a.max_levels = kMaxLevels;
  // a range the CTAs can hold on chip needs only as many CTAs as it fills
  uint64_t grid = cfg.grid;
  const uint64_t need = (body_end - h + Coop<T, KV>::Keys - 1) / Coop<T, KV>::Keys;
  if (need < grid) grid = need ? need : 1;
  // a body the CTAs hold at level 0 is finished on chip: no handoff can occur
  const bool handoff = handoff_var != nullptr && need > grid;
  a.handoff = handoff ? 1 : 0;
  a.level_cap = (level_cap >= 1 && level_cap < (uint32_t)kMaxLevels) ? (int)level_cap
                                                                     : kMaxLevels - 1;
  if (cfg.events) cudaEventRecord(cfg.events[0], st);
  cudaError_t e = launch_cooperative(partition_kernel<T, KV>, (uint32_t)grid, R::Threads, smem,
                                     st, keys, vals, a, S);
  cfg.launches++;
  if (cfg.events) cudaEventRecord(cfg.events[1], st);
  if (e != cudaSuccess) return e;
  if (handoff) {  // the range handed over, if any (an empty one returns at once)
    e = launch_lowspace<T, KV>(keys, vals, 0, 0, body_end - h, S.handoff, pivot, kHandoffBlock,
                               ~0ull, handoff_var, S, nullptr, cfg);
    if (e != cudaSuccess) return e;
  }
  finalize_kernel<T, KV><<<1, 32, 0, st>>>(keys, vals, n, h, body_end, pivot, S);
  cfg.launches++;
  return cudaGetLastError();
}

template <typename T, bool KV>
cudaError_t launch_first_level(T* keys, uint64_t* vals, uint64_t n, T pivot, uint64_t seed,
                               int strided, const TaskScratch& S, LaunchCfg& cfg, uint64_t* hp,
                               uint64_t* body_endp) {
  using R = Tr<T, KV>;
  cudaStream_t st = cfg.stream;
  const size_t smem = stream_smem_bytes<T, KV>();
  desc_init_kernel<<<1, 32, 0, st>>>(S);
  cfg.launches++;
  const uintptr_t addr = reinterpret_cast<uintptr_t>(keys);
  const uint64_t h = ((16 - (addr & 15)) & 15) / R::K;
  const uint64_t body_end = h + ((n - h) / R::A) * R::A;
  *hp = h;
  *body_endp = body_end;
  PartArgs a;
  a.body_lo = h;
  a.body_hi = body_end;
  a.pivot = (uint64_t)pivot;
  a.seed = seed;
  a.strided = strided;
  a.max_levels = 1;
  a.handoff = 0;
  a.level_cap = kMaxLevels - 1;
  uint64_t grid = cfg.grid;
  const uint64_t need = (body_end - h + Coop<T, KV>::Keys - 1) / Coop<T, KV>::Keys;
  if (need < grid) grid = need ? need : 1;
  if (cfg.events) cudaEventRecord(cfg.events[0], st);
  cudaError_t e = launch_cooperative(partition_kernel<T, KV>, (uint32_t)grid, R::Threads, smem,
                                     st, keys, vals, a, S);
  cfg.launches++;
  if (cfg.events) cudaEventRecord(cfg.events[1], st);
  return e;
}

template <typename T, bool KV>
cudaError_t launch_finalize(T* keys, uint64_t* vals, uint64_t n, uint64_t h, uint64_t body_end,
                            T pivot, const TaskScratch& S, LaunchCfg& cfg) {
  finalize_kernel<T, KV><<<1, 32, 0, cfg.stream>>>(keys, vals, n, h, body_end, pivot, S);
  cfg.launches++;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_step(T* keys, uint64_t n, T pivot, uint64_t b, uint64_t g, uint64_t seed,
                        uint64_t level, int strided, const TaskScratch& S, LaunchCfg& cfg) {
  cudaStream_t st = cfg.stream;
  desc_init_kernel<<<1, 32, 0, st>>>(S);
  cfg.launches++;
  LevelArgs a;
  a.lo = 0;
  a.hi = n;
  a.body_lo = 0;
  a.body_hi = n;
  a.pivot = (uint64_t)pivot;
  a.seed = seed;
  a.level = level;
  a.fixed_b = b;
  a.fixed_g = g;
  a.strided = strided;
  a.force_finish = 0;
  level_kernel<T, false><<<cfg.grid, Tr<T, false>::Threads, stream_smem_bytes<T, false>(), st>>>(
      keys, nullptr, a, S.desc, S.status);
  cfg.launches++;
  return cudaGetLastError();
}

// ------------------------------------------------------------ fill kernels
__global__ void fill_u64_kernel(uint64_t* d, uint64_t n, uint64_t seed) {
  for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < n;
       q += (uint64_t)gridDim.x * blockDim.x)
    d[q] = sm_stream(seed, q);
}
__global__ void fill_u32_kernel(uint32_t* d, uint64_t n, uint64_t seed) {
  for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < n;
       q += (uint64_t)gridDim.x * blockDim.x)
    d[q] = (uint32_t)sm_stream(seed, q);
}
__global__ void iota_u64_kernel(uint64_t* d, uint64_t n) {
  for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < n;
       q += (uint64_t)gridDim.x * blockDim.x)
    d[q] = q;
}

static unsigned fill_blocks(uint64_t n) {
  uint64_t b = (n + 255) / 256;
  return (unsigned)(b < 4096 ? (b ? b : 1) : 4096);
}

cudaError_t launch_fill_u64(uint64_t* d, uint64_t n, uint64_t seed, cudaStream_t s) {
  fill_u64_kernel<<<fill_blocks(n), 256, 0, s>>>(d, n, seed);
  return cudaGetLastError();
}
cudaError_t launch_fill_u32(uint32_t* d, uint64_t n, uint64_t seed, cudaStream_t s) {
  fill_u32_kernel<<<fill_blocks(n), 256, 0, s>>>(d, n, seed);
  return cudaGetLastError();
}
cudaError_t launch_iota_u64(uint64_t* d, uint64_t n, cudaStream_t s) {
  iota_u64_kernel<<<fill_blocks(n), 256, 0, s>>>(d, n);
  return cudaGetLastError();
}

// explicit instantiations
template cudaError_t streaming_grid<uint64_t, false>(int, uint32_t*);
template cudaError_t streaming_grid<uint32_t, false>(int, uint32_t*);
template cudaError_t streaming_grid<uint64_t, true>(int, uint32_t*);
#define LP_INST_SMOOTHED(T, KV)                                                               \
  template cudaError_t launch_smoothed<T, KV>(T*, uint64_t*, uint64_t, T, uint64_t, int,          \
                                              const TaskScratch&, LaunchCfg&, void*, uint32_t);   \
  template bool smoothed_may_hand_off<T, KV>(uint64_t, uint32_t);
LP_INST_SMOOTHED(uint64_t, false)
LP_INST_SMOOTHED(uint32_t, false)
LP_INST_SMOOTHED(uint64_t, true)
#undef LP_INST_SMOOTHED
#define LP_INST_FIRST(T, KV)                                                                  \
  template cudaError_t launch_first_level<T, KV>(T*, uint64_t*, uint64_t, T, uint64_t, int,       \
                                                 const TaskScratch&, LaunchCfg&, uint64_t*,       \
                                                 uint64_t*);                                      \
  template cudaError_t launch_finalize<T, KV>(T*, uint64_t*, uint64_t, uint64_t, uint64_t, T,    \
                                              const TaskScratch&, LaunchCfg&);
LP_INST_FIRST(uint64_t, false)
LP_INST_FIRST(uint32_t, false)
LP_INST_FIRST(uint64_t, true)
#undef LP_INST_FIRST
template cudaError_t launch_step<uint64_t>(uint64_t*, uint64_t, uint64_t, uint64_t, uint64_t,
                                           uint64_t, uint64_t, int, const TaskScratch&,
                                           LaunchCfg&);
template cudaError_t launch_step<uint32_t>(uint32_t*, uint64_t, uint32_t, uint64_t, uint64_t,
                                           uint64_t, uint64_t, int, const TaskScratch&,
                                           LaunchCfg&);

}  // namespace lp
