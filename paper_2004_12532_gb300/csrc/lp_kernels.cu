// lp_kernels.cu -- kernels of the Recursive Smoothed Striding partition
// (Sec. 4 of arXiv 2004.12532) and their host launchers.
//
//   desc_init_kernel     resets the per-level descriptors and the status word
//   level_kernel         one Partial Partition Step over the range the previous
//                        level left open ([v_min, v_max) of Sec. 4), with the
//                        parameter rule of lp_plan.h; a range small enough runs
//                        as one group, i.e. the paper's base case
//   finalize_kernel      places the (< 16-byte) unaligned head and tail keys
//                        and writes the split t
//   small_kernel         whole partition of a short array in one CTA
//   fill kernels         seeded synthetic inputs (SplitMix64), harness only
#include <cuda_runtime.h>
#include <stdint.h>

#include "lp_launch.h"
#include "lp_smoothed.cuh"

namespace lp {

size_t level_desc_bytes() { return sizeof(LevelDesc); }

__global__ void desc_init_kernel(LevelDesc* d, int count, uint32_t* status) {
  int t = threadIdx.x;
  if (t < count) {
    d[t].vmin = ~0ull;
    d[t].vmax = 0ull;
    d[t].count = 0ull;
    d[t].lo = d[t].hi = d[t].b = d[t].g = d[t].pad = 0ull;
  }
  if (t == 0) *status = 0u;
}

// Range of a level: the caller's range at level 0, else the previous level's
// [v_min, v_max).  Extended outward to 16-byte boundaries of the body: keys
// added on the left are already predecessors in final position and keys added
// on the right successors, so partitioning the wider range is equivalent.
__device__ __forceinline__ bool level_range(const LevelArgs& a, const LevelDesc* in,
                                            uint32_t A, uint64_t& lo, uint64_t& hi) {
  if (in) {
    lo = in->vmin;
    hi = in->vmax;
    if (lo >= hi) return false;
  } else {
    lo = a.lo;
    hi = a.hi;
    if (lo >= hi) return false;
  }
  lo = a.body_lo + ((lo - a.body_lo) / A) * A;
  uint64_t h2 = a.body_lo + ((hi - a.body_lo + A - 1) / A) * A;
  hi = h2 < a.body_hi ? h2 : a.body_hi;
  return lo < hi;
}

template <typename T, bool KV>
__global__ void __launch_bounds__(Tr<T, KV>::Threads) level_kernel(T* keys, uint64_t* vals,
                                                                   LevelArgs a,
                                                                   const LevelDesc* in,
                                                                   LevelDesc* out,
                                                                   uint32_t* status) {
  using R = Tr<T, KV>;
  extern __shared__ __align__(128) unsigned char smem_raw[];

  uint64_t lo, hi;
  if (!level_range(a, in, R::A, lo, hi)) return;
  const uint64_t n = hi - lo;
  const uint64_t total_warps = (uint64_t)gridDim.x * R::Warps;

  uint64_t b, g;
  if (a.fixed_b) {
    b = a.fixed_b;
    g = a.fixed_g;
  } else {
    const StepParams P = choose_params(n, R::K, total_warps, R::LineBytes, R::FinishKeys);
    b = P.b;
    g = P.g;
    if (a.force_finish && g != 0) g = 1;  // last level: one group takes the rest
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    out->lo = lo; out->hi = hi; out->b = b; out->g = g;
  }
  if (g == 0) {
    // the paper's base case: one CTA partitions the range in shared memory
    if (blockIdx.x != 0) return;
    const uint32_t cnt = cta_partition_smem<T, KV>(keys + lo, KV ? vals + lo : nullptr,
                                                   (uint32_t)n, (T)a.pivot, smem_raw);
    if (threadIdx.x == 0) {
      out->vmin = lo + cnt;
      out->vmax = lo + cnt;
      out->count = cnt;
    }
    return;
  }

  const StepGeom G = make_geom(n, b, g, level_seed(a.seed, a.level), a.strided);
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const uint64_t gw = (uint64_t)blockIdx.x * R::Warps + warp;
  if (gw >= G.g) return;  // warps are independent: no CTA barrier below
  WarpSmem<T, KV>& ws = reinterpret_cast<WarpSmem<T, KV>*>(smem_raw)[warp];
  if (lane == 0) {
    for (uint32_t s = 0; s < kStages; s++) mbar_init(&ws.bar[s], 1);
    fence_mbar_init();
    fence_proxy_async_smem();
  }
  __syncwarp();

  uint32_t phase = 0;
  T* base = keys + lo;
  uint64_t* vbase = KV ? vals + lo : nullptr;
  const T pivot = (T)a.pivot;
  for (uint64_t i = gw; i < G.g; i += total_warps) {
    const int64_t nl = (int64_t)group_num_lines(G, i);
    uint64_t k = 0;
    if (!warp_pair_group<T, KV>(base, vbase, G, i, nl, pivot, ws, phase, k, status)) break;
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
// final split t; there are at most a dozen, and one thread swaps them.
template <typename T, bool KV>
__global__ void finalize_kernel(T* keys, uint64_t* vals, uint64_t n, uint64_t h,
                                uint64_t body_end, T pivot, const LevelDesc* d0,
                                const LevelDesc* dlast, uint32_t* status, uint64_t* split) {
  if (threadIdx.x != 0) return;
  if (dlast->vmin < dlast->vmax) atomicOr(status, kStatUnfinished);
  const uint64_t cb = d0->count;
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
    atomicOr(status, kStatRing);
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
  *split = t;
}

uint64_t small_limit(uint32_t key_bytes, bool kv) {
  return kFinishBytes / (key_bytes + (kv ? 8u : 0u));
}

// Whole partition of an array of n <= small_limit keys in one CTA.
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
  e = cudaFuncSetAttribute(level_kernel<T, KV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(small_kernel<T, KV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  if (e != cudaSuccess) return e;
  int sms = 0, per = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, level_kernel<T, KV>,
                                                    Tr<T, KV>::Threads, smem);
  if (e != cudaSuccess) return e;
  if (per < 1) per = 1;
  *grid = (uint32_t)(sms * per);
  return cudaSuccess;
}

template <typename T, bool KV>
cudaError_t launch_smoothed(T* keys, uint64_t* vals, uint64_t n, T pivot, uint64_t seed,
                            int strided, const TaskScratch& S, LaunchCfg& cfg) {
  using R = Tr<T, KV>;
  cudaStream_t st = cfg.stream;
  if (n <= small_limit(R::K, KV)) {
    const size_t smem = stream_smem_bytes<T, KV>();
    if (cfg.level_events)
      for (int L = 0; L <= kMaxLevels; L++) cudaEventRecord(cfg.level_events[L], st);
    small_kernel<T, KV><<<1, R::Threads, smem, st>>>(keys, vals, (uint32_t)n, pivot, S.split);
    cfg.launches++;
    desc_init_kernel<<<1, 32, 0, st>>>(S.desc, kMaxLevels, S.status);
    cfg.launches++;
    return cudaGetLastError();
  }
  const uintptr_t addr = reinterpret_cast<uintptr_t>(keys);
  const uint64_t h = ((16 - (addr & 15)) & 15) / R::K;
  const uint64_t body_end = h + ((n - h) / R::A) * R::A;
  const size_t smem = stream_smem_bytes<T, KV>();

  desc_init_kernel<<<1, 32, 0, st>>>(S.desc, kMaxLevels, S.status);
  cfg.launches++;
  for (int L = 0; L < kMaxLevels; L++) {
    LevelArgs a;
    a.lo = h;
    a.hi = body_end;
    a.body_lo = h;
    a.body_hi = body_end;
    a.pivot = (uint64_t)pivot;
    a.seed = seed;
    a.level = (uint64_t)L;
    a.fixed_b = 0;
    a.fixed_g = 0;
    a.strided = (strided && L == 0) ? 1 : 0;
    a.force_finish = (L == kMaxLevels - 1) ? 1 : 0;
    const LevelDesc* in = L ? S.desc + (L - 1) : nullptr;
    if (cfg.level_events) cudaEventRecord(cfg.level_events[L], st);
    level_kernel<T, KV><<<cfg.grid, R::Threads, smem, st>>>(keys, vals, a, in, S.desc + L,
                                                            S.status);
    cfg.launches++;
  }
  if (cfg.level_events) cudaEventRecord(cfg.level_events[kMaxLevels], st);
  finalize_kernel<T, KV><<<1, 32, 0, st>>>(keys, vals, n, h, body_end, pivot, S.desc,
                                           S.desc + (kMaxLevels - 1), S.status, S.split);
  cfg.launches++;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_step(T* keys, uint64_t n, T pivot, uint64_t b, uint64_t g, uint64_t seed,
                        uint64_t level, int strided, const TaskScratch& S, LaunchCfg& cfg) {
  cudaStream_t st = cfg.stream;
  desc_init_kernel<<<1, 32, 0, st>>>(S.desc, kMaxLevels, S.status);
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
      keys, nullptr, a, nullptr, S.desc, S.status);
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
template cudaError_t launch_smoothed<uint64_t, false>(uint64_t*, uint64_t*, uint64_t, uint64_t,
                                                      uint64_t, int, const TaskScratch&,
                                                      LaunchCfg&);
template cudaError_t launch_smoothed<uint32_t, false>(uint32_t*, uint64_t*, uint64_t, uint32_t,
                                                      uint64_t, int, const TaskScratch&,
                                                      LaunchCfg&);
template cudaError_t launch_smoothed<uint64_t, true>(uint64_t*, uint64_t*, uint64_t, uint64_t,
                                                     uint64_t, int, const TaskScratch&,
                                                     LaunchCfg&);
template cudaError_t launch_step<uint64_t>(uint64_t*, uint64_t, uint64_t, uint64_t, uint64_t,
                                           uint64_t, uint64_t, int, const TaskScratch&,
                                           LaunchCfg&);
template cudaError_t launch_step<uint32_t>(uint32_t*, uint64_t, uint32_t, uint64_t, uint64_t,
                                           uint64_t, uint64_t, int, const TaskScratch&,
                                           LaunchCfg&);

}  // namespace lp
