// lp_lowspace.cu -- the Blocked-Prefix-Sum partition (Sec. 3 of arXiv
// 2004.12532, figures "Blocked-Prefix-Sum Partition Algorithm"), with the
// prefix values stored explicitly as the paper's low-space implementation
// does (Sec. 5): ⌊n/B⌋ counters, 8 bytes each, B = 4096 by default (1/4096 of
// the keys' count, 0.024% of a uint64 array's bytes).
//
// One cooperative launch runs the phases with grid barriers between them:
//   1. count the predecessors; when they are the majority, swap the roles and
//      work on the logically reversed array (ParallelPartition's role swap);
//   2. MakeSuccessorHeavy (Lemma 3.1): for i < floor(m/2) swap A[i] and
//      A[m-1-i] when the first is a predecessor and the second a successor,
//      then m <- ceil(m/2); small levels run inside one CTA;
//   3. block counts and their prefix: v[i] = predecessors in blocks 0..i
//      (blocks of B keys, the last block takes the remainder);
//   4. Reorder (Lemma "Reordering phase"): the prefixes P_0 ⊃ P_1 ⊃ ... with
//      P_{j+1} the smallest prefix of whole blocks holding 4/5 of P_j; the
//      innermost prefix (at most base_keys, or the paper's 5B) is partitioned
//      on chip; then, from the inside out, every predecessor of a block beyond
//      P_{j+1} is swapped with position v[i-1] + (its rank in the block), a
//      successor inside P_{j+1} -- conflict-free because P_{j+1} is
//      successor-heavy; one warp per block, its rounds of 32 keys ranked by
//      ballots.
// Every load of keys that another CTA may have written goes through L2
// (ld.global.cg), so no CTA reads a stale L1 line after a barrier.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lp_coop.cuh"
#include "lp_launch.h"

namespace lp {

namespace {

constexpr uint32_t kLT = 256;               // threads per CTA
constexpr uint64_t kMshSmall = 1u << 15;    // pair counts below this: one CTA
constexpr uint32_t kUnroll = 8;             // independent loads in flight per thread
constexpr int kMaxReorderLevels = 96;

struct LowArgs {
  uint64_t lo, hi;                 // range, unless range_desc is set
  const LevelDesc* range_desc;     // range = [vmin, vmax) of this descriptor
  uint64_t pivot;
  uint64_t B;                      // block size
  uint64_t base_keys;              // innermost prefix finished on chip at this size
  uint64_t* v;                     // nb prefix counters
  uint64_t nb_cap;                 // counters the scratch holds
  unsigned long long* cta;         // one word per CTA
  unsigned long long* total;       // predecessor count of the range
  uint64_t* split;                 // if set: the split (count) is written here
  unsigned long long* tl;          // device timestamps: start, then the end of each phase
};

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) {
  if constexpr (sizeof(T) == 8) return (T)__ldcg(reinterpret_cast<const unsigned long long*>(p));
  else return (T)__ldcg(reinterpret_cast<const unsigned int*>(p));
}

// CTA-wide sum (all threads call; result in every thread)
__device__ __forceinline__ unsigned long long cta_sum(unsigned long long x,
                                                      unsigned long long* red) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  __syncthreads();
  if (lane == 0) red[warp] = x;
  __syncthreads();
  unsigned long long s = 0;
  for (uint32_t w = 0; w < kLT / 32; w++) s += red[w];
  return s;
}

template <typename T, bool KV>
__global__ void __launch_bounds__(kLT, 2) lowspace_kernel(T* keys, uint64_t* vals, LowArgs a,
                                                       TaskScratch S) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ unsigned int flag;
  __shared__ unsigned long long red[kLT / 32];
  __shared__ uint64_t levM[kMaxReorderLevels], levT[kMaxReorderLevels], levNB[kMaxReorderLevels];
  __shared__ int nlev;
  __shared__ uint64_t mbase_s;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint64_t gtid = (uint64_t)blockIdx.x * kLT + tid, gstride = (uint64_t)gridDim.x * kLT;
  const bool leader = blockIdx.x == 0 && tid == 0;
  auto fail = [&]() {
    if (tid == 0) atomicOr(S.status, kStatTimeout);
  };

  uint64_t lo = a.lo, hi = a.hi;
  if (a.range_desc) {
    lo = __ldcg(&a.range_desc->vmin);
    hi = __ldcg(&a.range_desc->vmax);
    if (lo >= hi) { lo = 0; hi = 0; }
  }
  const uint64_t n = hi - lo;
  T* A = keys + lo;
  uint64_t* Y = KV ? vals + lo : nullptr;
  const T pivot = (T)a.pivot;
  auto stamp = [&](int k) {
    if (leader) a.tl[k] = global_timer_ns();
  };
  stamp(0);

  // ---- 1. count, role swap
  {
    unsigned long long c = 0;
    for (uint64_t q0 = gtid; q0 < n; q0 += kUnroll * gstride) {  // kUnroll loads in flight
      T x[kUnroll];
#pragma unroll
      for (uint32_t u = 0; u < kUnroll; u++) {
        const uint64_t q = q0 + u * gstride;
        x[u] = q < n ? ldcg(&A[q]) : pivot;
      }
#pragma unroll
      for (uint32_t u = 0; u < kUnroll; u++)
        c += (q0 + u * gstride < n && x[u] <= pivot) ? 1u : 0u;
    }
    c = cta_sum(c, red);
    if (tid == 0) atomicAdd(a.total, c);
  }
  if (!grid_barrier(S.bar, gridDim.x, &flag)) { fail(); return; }
  const uint64_t cnt = __ldcg(a.total);
  if (leader && a.split) *a.split = cnt;
  stamp(1);
  if (n < 2) return;
  const bool flip = 2 * (n - cnt) < n;
  auto mem = [&](uint64_t i) -> uint64_t { return flip ? n - 1 - i : i; };
  auto isp = [&](T x) -> bool { return flip ? (x > pivot) : (x <= pivot); };
  auto swap_at = [&](uint64_t p, uint64_t q, T x, T y) {
    A[p] = y;
    A[q] = x;
    if constexpr (KV) {
      const uint64_t u = ldcg(&Y[p]), w = ldcg(&Y[q]);
      Y[p] = w;
      Y[q] = u;
    }
  };

  // ---- 2. MakeSuccessorHeavy
  uint64_t m = n;
  while (m > 1) {
    const uint64_t half = m / 2;
    if (half >= kMshSmall) {
      for (uint64_t i0 = gtid; i0 < half; i0 += kUnroll * gstride) {
        T x[kUnroll], y[kUnroll];
#pragma unroll
        for (uint32_t u = 0; u < kUnroll; u++) {
          const uint64_t i = i0 + u * gstride;
          if (i < half) { x[u] = ldcg(&A[mem(i)]); y[u] = ldcg(&A[mem(m - 1 - i)]); }
        }
#pragma unroll
        for (uint32_t u = 0; u < kUnroll; u++) {
          const uint64_t i = i0 + u * gstride;
          if (i < half && isp(x[u]) && !isp(y[u])) swap_at(mem(i), mem(m - 1 - i), x[u], y[u]);
        }
      }
      if (!grid_barrier(S.bar, gridDim.x, &flag)) { fail(); return; }
      m -= half;
    } else {
      if (blockIdx.x == 0) {
        while (m > 1) {
          const uint64_t h2 = m / 2;
          for (uint64_t i = tid; i < h2; i += kLT) {
            const uint64_t p = mem(i), q = mem(m - 1 - i);
            const T x = ldcg(&A[p]), y = ldcg(&A[q]);
            if (isp(x) && !isp(y)) swap_at(p, q, x, y);
          }
          __syncthreads();
          m -= h2;
        }
      }
      m = 1;
      if (!grid_barrier(S.bar, gridDim.x, &flag)) { fail(); return; }
    }
  }

  stamp(2);

  // ---- 3. block prefix v[i]
  const uint64_t B = a.B;
  const uint64_t nb = n / B;
  if (nb > a.nb_cap) {  // never expected: the host sizes the scratch for the array
    if (tid == 0) atomicOr(S.status, kStatRing);
    return;
  }
  if (nb > 0) {
    const uint64_t bpc = (nb + gridDim.x - 1) / gridDim.x;
    const uint64_t b0 = min((uint64_t)blockIdx.x * bpc, nb), b1 = min(b0 + bpc, nb);
    unsigned long long run = 0;
    for (uint64_t b = b0; b < b1; b++) {
      const uint64_t s = b * B, e = (b + 1 == nb) ? n : s + B;
      unsigned long long c = 0;
      for (uint64_t q0 = s + tid; q0 < e; q0 += (uint64_t)kUnroll * kLT) {
        T x[kUnroll];
#pragma unroll
        for (uint32_t u = 0; u < kUnroll; u++) {
          const uint64_t q = q0 + (uint64_t)u * kLT;
          if (q < e) x[u] = ldcg(&A[mem(q)]);
        }
#pragma unroll
        for (uint32_t u = 0; u < kUnroll; u++)
          c += (q0 + (uint64_t)u * kLT < e && isp(x[u])) ? 1u : 0u;
      }
      c = cta_sum(c, red);
      run += c;
      if (tid == 0) __stcg(reinterpret_cast<unsigned long long*>(&a.v[b]), run);
    }
    if (tid == 0) __stcg(&a.cta[blockIdx.x], run);
    if (!grid_barrier(S.bar, gridDim.x, &flag)) { fail(); return; }
    unsigned long long off = 0;
    for (uint32_t c2 = tid; c2 < blockIdx.x; c2 += kLT) off += __ldcg(&a.cta[c2]);
    off = cta_sum(off, red);
    for (uint64_t b = b0 + tid; b < b1; b += kLT) {
      unsigned long long* pv = reinterpret_cast<unsigned long long*>(&a.v[b]);
      __stcg(pv, __ldcg(pv) + off);
    }
    if (!grid_barrier(S.bar, gridDim.x, &flag)) { fail(); return; }
  }

  stamp(3);

  // ---- 4. Reorder: the prefix levels, innermost first
  if (tid == 0) {
    int j = 0;
    uint64_t mm = n, nbj = nb;
    for (;;) {
      const uint64_t t = (4 * mm + 5 * B - 1) / (5 * B);  // least t with t B >= 4 mm / 5
      if (mm <= a.base_keys || mm <= 5 * B || t >= nbj || j == kMaxReorderLevels) break;
      levM[j] = mm;
      levT[j] = t;
      levNB[j] = nbj;
      j++;
      mm = t * B;
      nbj = t;
    }
    nlev = j;
    mbase_s = mm;  // the innermost prefix
  }
  __syncthreads();
  const int L = nlev;
  const uint64_t mbase = mbase_s;
  {
    // the innermost prefix, partitioned on chip: in memory it is [0, mbase)
    // or, for the reversed view, [n - mbase, n) with the roles back in place
    const uint64_t off = flip ? n - mbase : 0;
    const uint64_t t = coop_finish<T, KV>(A + off, KV ? Y + off : nullptr, mbase, pivot, S,
                                          smem_raw, &flag);
    if (t == ~0ull) { fail(); return; }
    if (!grid_barrier(S.bar, gridDim.x, &flag)) { fail(); return; }
  }
  stamp(4);
  // Reorder level by level, outward; one warp per block, kUnroll rounds of 32
  // keys in flight: every predecessor of block i goes to v[i-1] + its rank in
  // the block (a successor inside the successor-heavy prefix), so the target
  // loads of a group of rounds can all be issued before its stores
  const uint64_t gwarp = ((uint64_t)blockIdx.x * kLT + tid) >> 5;
  const uint64_t nwarps = gstride >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  for (int j = L - 1; j >= 0; j--) {
    const uint64_t M = levM[j], t0 = levT[j], NB = levNB[j];
    for (uint64_t i = t0 + gwarp; i < NB; i += nwarps) {
      const uint64_t s0 = i * B, e = (i + 1 == NB) ? M : s0 + B;
      uint64_t y = __ldcg(reinterpret_cast<const unsigned long long*>(&a.v[i - 1]));
      for (uint64_t r0 = s0; r0 < e; r0 += 32ull * kUnroll) {
        T x[kUnroll], z[kUnroll];
        uint64_t tg[kUnroll];
        uint32_t f = 0, bal[kUnroll];
#pragma unroll
        for (uint32_t u = 0; u < kUnroll; u++) {
          const uint64_t q = r0 + 32ull * u + lane;
          if (q < e) {
            x[u] = ldcg(&A[mem(q)]);
            f |= (isp(x[u]) ? 1u : 0u) << u;
          }
        }
        uint32_t run = 0;
#pragma unroll
        for (uint32_t u = 0; u < kUnroll; u++) {
          bal[u] = __ballot_sync(0xffffffffu, (f >> u) & 1u);
          if ((f >> u) & 1u) {
            tg[u] = mem(y + run + __popc(bal[u] & lt));
            z[u] = ldcg(&A[tg[u]]);
          }
          run += __popc(bal[u]);
        }
#pragma unroll
        for (uint32_t u = 0; u < kUnroll; u++)
          if ((f >> u) & 1u) swap_at(tg[u], mem(r0 + 32ull * u + lane), z[u], x[u]);
        y += run;
      }
    }
    if (!grid_barrier(S.bar, gridDim.x, &flag)) { fail(); return; }
  }
  stamp(5);
}

}  // namespace

size_t lowspace_scratch_bytes(uint64_t n, uint64_t B, uint32_t grid) {
  const uint64_t nb = B ? n / B : 0;
  return ((nb + 1) * 8 + 255) / 256 * 256 + ((size_t)grid * 8 + 255) / 256 * 256 + 256 + 256;
}

template <typename T, bool KV>
cudaError_t launch_lowspace(T* keys, uint64_t* vals, uint64_t lo, uint64_t hi, uint64_t n_cap,
                            const LevelDesc* range_desc, T pivot, uint64_t B, uint64_t base_keys,
                            void* var, const TaskScratch& S, uint64_t* split, LaunchCfg& cfg) {
  cudaStream_t st = cfg.stream;
  // the scratch is laid out for the largest range it may see (the range may
  // only be known on the device)
  const uint64_t nb = B ? n_cap / B : 0;
  unsigned char* p = static_cast<unsigned char*>(var);
  LowArgs a;
  a.lo = lo;
  a.hi = hi;
  a.range_desc = range_desc;
  a.pivot = (uint64_t)pivot;
  a.B = B;
  a.v = reinterpret_cast<uint64_t*>(p);
  a.nb_cap = nb;
  p += ((nb + 1) * 8 + 255) / 256 * 256;
  a.cta = reinterpret_cast<unsigned long long*>(p);
  p += ((size_t)cfg.grid * 8 + 255) / 256 * 256;
  a.total = reinterpret_cast<unsigned long long*>(p);
  a.tl = reinterpret_cast<unsigned long long*>(p + 256);
  a.split = split;
  const size_t smem = level_smem_bytes<T, KV>();
  cudaError_t e = cudaFuncSetAttribute(lowspace_kernel<T, KV>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // a cooperative grid must fit on the device at once: size it by this kernel
  int dev = 0, sms = 0, per = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, lowspace_kernel<T, KV>, kLT,
                                                         smem)) != cudaSuccess)
    return e;
  uint32_t grid = cfg.grid;
  if ((uint64_t)sms * (uint64_t)(per < 1 ? 1 : per) < grid) grid = (uint32_t)(sms * (per < 1 ? 1 : per));
  const uint64_t cap = (uint64_t)grid * Coop<T, KV>::Keys;
  a.base_keys = base_keys < cap ? base_keys : cap;
  if (a.base_keys < 5 * B) a.base_keys = 0;  // the paper's base case decides
  e = cudaMemsetAsync(a.total, 0, 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.tl, 0, 8 * kLowPhases, st);
  if (e != cudaSuccess) return e;
  if (cfg.phase_stamps) *cfg.phase_stamps = a.tl;
  e = launch_cooperative(lowspace_kernel<T, KV>, grid, kLT, smem, st, keys, vals, a, S);
  cfg.launches++;
  return e;
}

template cudaError_t launch_lowspace<uint64_t, false>(uint64_t*, uint64_t*, uint64_t, uint64_t,
                                                      uint64_t, const LevelDesc*, uint64_t, uint64_t,
                                                      uint64_t, void*, const TaskScratch&,
                                                      uint64_t*, LaunchCfg&);
template cudaError_t launch_lowspace<uint32_t, false>(uint32_t*, uint64_t*, uint64_t, uint64_t,
                                                      uint64_t, const LevelDesc*, uint32_t, uint64_t,
                                                      uint64_t, void*, const TaskScratch&,
                                                      uint64_t*, LaunchCfg&);
template cudaError_t launch_lowspace<uint64_t, true>(uint64_t*, uint64_t*, uint64_t, uint64_t,
                                                     uint64_t, const LevelDesc*, uint64_t, uint64_t,
                                                     uint64_t, void*, const TaskScratch&,
                                                     uint64_t*, LaunchCfg&);

}  // namespace lp
