// lp_coop.cuh -- the on-chip base case shared by the partition kernels: a
// range that fits in the shared memory of all co-resident CTAs is read once,
// counted, and written once to its final places after one grid barrier.
#pragma once
#include "lp_device.cuh"
#include "lp_launch.h"
#include "lp_smoothed.cuh"

namespace lp {

template <typename T, bool KV>
struct Coop {
  // keys one CTA holds in the on-chip base case (a multiple of the 16-byte
  // alignment unit), and the shared memory it uses
  static constexpr size_t SmemBytes = level_smem_bytes<T, KV>();
  static constexpr uint32_t Keys =
      (uint32_t)((SmemBytes - 256) / (sizeof(T) + (KV ? 8 : 0))) / Tr<T, KV>::A * Tr<T, KV>::A;
};

// The base case on chip: the range base[0..n) is split into gridDim.x blocks
// of B keys; every CTA stages its block in shared memory and counts its
// predecessors; after a grid barrier each CTA knows the predecessors of the
// blocks before it and writes its predecessors, then its successors, to their
// final places (stable).  Every key is read once and written once.  All threads
// of all CTAs call this, and a CTA has exactly NT threads (the per-warp sums
// take 3 * NT/32 words).  Returns the predecessor count of the range, or ~0
// if this CTA gave up at the grid barrier or was launched with another
// thread count.
template <typename T, bool KV, uint32_t NT = Tr<T, KV>::Threads>
__device__ uint64_t coop_finish(T* __restrict__ base, uint64_t* __restrict__ vbase, uint64_t n,
                                T pivot, const TaskScratch& S, unsigned char* smem,
                                unsigned int* flag) {
  constexpr uint32_t A = Tr<T, KV>::A;
  static_assert(NT % 32 == 0 && 3 * (NT / 32) * 4 <= 128, "per-warp sums fit 128 bytes");
  if (blockDim.x != NT) {  // same in every CTA: all of them leave here
    if (threadIdx.x == 0) atomicOr(S.status, kStatRing);
    return ~0ull;
  }
  uint32_t* wsum = reinterpret_cast<uint32_t*>(smem);  // 3 * NT/32 words
  T* sk = reinterpret_cast<T*>(smem + 128);
  uint64_t* sv = reinterpret_cast<uint64_t*>(smem + 128 + (size_t)Coop<T, KV>::Keys * sizeof(T));
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  uint64_t B = (n + gridDim.x - 1) / gridDim.x;
  B = (B + A - 1) / A * A;
  const uint64_t s0 = min((uint64_t)blockIdx.x * B, n), s1 = min(s0 + B, n);
  const uint32_t m = (uint32_t)(s1 - s0);
  for (uint32_t q = tid; q < m; q += NT) {  // through L2: other CTAs wrote these
    if constexpr (sizeof(T) == 8)
      sk[q] = (T)__ldcg(reinterpret_cast<const unsigned long long*>(base + s0 + q));
    else
      sk[q] = (T)__ldcg(reinterpret_cast<const unsigned int*>(base + s0 + q));
    if constexpr (KV) sv[q] = __ldcg(reinterpret_cast<const unsigned long long*>(vbase + s0 + q));
  }
  __syncthreads();
  const uint32_t per = (m + NT - 1) / NT;
  const uint32_t q0 = min(m, tid * per), q1 = min(m, q0 + per);
  uint32_t cnt = 0;
  for (uint32_t q = q0; q < q1; q++) cnt += sk[q] <= pivot;
  uint32_t incl = cnt;
#pragma unroll
  for (uint32_t o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  uint32_t wb = 0, tot = 0;
  for (uint32_t w = 0; w < NT / 32; w++) {
    wb += w < warp ? wsum[w] : 0u;
    tot += wsum[w];
  }
  if (tid == 0) S.counts[blockIdx.x] = tot;
  if (!grid_barrier(S.bar, gridDim.x, flag)) return ~0ull;
  // predecessors before this block, and in the whole range
  uint32_t before = 0, all = 0;
  for (uint32_t c = tid; c < gridDim.x; c += NT) {
    const uint32_t v = __ldcg(&S.counts[c]);
    all += v;
    if (c < blockIdx.x) before += v;
  }
  before = __reduce_add_sync(0xffffffffu, before);
  all = __reduce_add_sync(0xffffffffu, all);
  if (lane == 0) { wsum[NT / 32 + warp] = before; wsum[2 * (NT / 32) + warp] = all; }
  __syncthreads();
  uint64_t bsum = 0, asum = 0;
  for (uint32_t w = 0; w < NT / 32; w++) {
    bsum += wsum[NT / 32 + w];
    asum += wsum[2 * (NT / 32) + w];
  }
  const uint32_t pre = wb + incl - cnt;  // predecessors before this thread's slice
  uint64_t pp = bsum + pre;
  uint64_t sp = asum + (s0 - bsum) + (q0 - pre);
  for (uint32_t q = q0; q < q1; q++) {
    const T x = sk[q];
    const uint64_t d = x <= pivot ? pp++ : sp++;
    base[d] = x;
    if constexpr (KV) vbase[d] = sv[q];
  }
  return asum;
}

}  // namespace lp
