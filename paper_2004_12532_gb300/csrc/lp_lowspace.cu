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
//      then m <- ceil(m/2); four levels per pass (three with payloads), each
//      thread holding one component of positions in registers, and the
//      passes below 2^16 keys inside one CTA;
//   3. block counts and their prefix: v[i] = predecessors in blocks 0..i
//      (blocks of B keys, the last block takes the remainder), one warp per
//      block, then a scan inside each CTA and across the CTAs;
//   4. Reorder (Lemma "Reordering phase"): the prefixes P_0 ⊃ P_1 ⊃ ... with
//      P_{j+1} the smallest prefix of whole blocks holding 4/5 of P_j; the
//      innermost prefix (at most base_keys, or the paper's 5B) is partitioned
//      on chip; then, from the inside out, every predecessor of a block beyond
//      P_{j+1} is swapped with position v[i-1] + (its rank in the block), a
//      successor inside P_{j+1} -- conflict-free because P_{j+1} is
//      successor-heavy; one warp per block, its rounds of 32 keys ranked by
//      ballots, the next round's keys loading while a round's targets do.
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
  uint64_t* split;                 // if set: the split (count) is written here
  unsigned long long* tl;          // device timestamps: start, then the end of each phase
  int prefix_only;                 // values kept in key order: stop after the prefix phase
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

// Predecessor count of the memory positions [p0, p1) of A, order being
// irrelevant: 16-byte loads (kUnroll per thread in flight) for the aligned
// body, single keys for the head and tail.  Thread `start` of `stride`
// threads takes its share; the caller sums the shares.
template <typename T, typename Isp>
__device__ __forceinline__ uint32_t count_span(const T* A, uint64_t p0, uint64_t p1,
                                               uint64_t start, uint64_t stride, const Isp& isp) {
  constexpr uint32_t E = 16 / sizeof(T);
  const uint64_t len = p1 - p0;
  uint64_t head = ((16u - ((uintptr_t)(A + p0) & 15u)) & 15u) / sizeof(T);
  if (head > len) head = len;
  const uint64_t nv = (len - head) / E;
  const uint4* vb = reinterpret_cast<const uint4*>(A + p0 + head);
  uint32_t c = 0;
  for (uint64_t v0 = start; v0 < nv; v0 += kUnroll * stride) {
    uint4 w[kUnroll];
#pragma unroll
    for (uint32_t u = 0; u < kUnroll; u++)
      if (v0 + u * stride < nv) w[u] = __ldcg(vb + v0 + u * stride);
#pragma unroll
    for (uint32_t u = 0; u < kUnroll; u++) {
      if (v0 + u * stride >= nv) continue;
      if constexpr (sizeof(T) == 8) {
        c += isp((T)(((uint64_t)w[u].y << 32) | w[u].x)) ? 1u : 0u;
        c += isp((T)(((uint64_t)w[u].w << 32) | w[u].z)) ? 1u : 0u;
      } else {
        c += (isp((T)w[u].x) ? 1u : 0u) + (isp((T)w[u].y) ? 1u : 0u) +
             (isp((T)w[u].z) ? 1u : 0u) + (isp((T)w[u].w) ? 1u : 0u);
      }
    }
  }
  const uint64_t t0 = p0 + head + nv * E, rest = head + (p1 - t0);
  for (uint64_t q = start; q < rest; q += stride)
    c += isp(ldcg(&A[q < head ? p0 + q : t0 + (q - head)])) ? 1u : 0u;
  return c;
}

// MakeSuccessorHeavy level k works on the prefix of m_k keys: it pairs i with
// m_k - 1 - i for i < h_k = floor(m_k / 2), and m_{k+1} = m_k - h_k.  Over L
// consecutive levels the positions fall into independent components: a root
// r < m_L, its level-(L-1) partner, their level-(L-2) partners, and so on, at
// most 2^L positions.  A pass loads one component into registers, applies the
// L levels' swaps in order and stores the positions that changed, so each
// position is read and written once per L levels instead of once per level.
template <bool KV>
constexpr int kMshFuse = KV ? 3 : 4;

template <int L>
__device__ __forceinline__ uint64_t msh_after(uint64_t m) {
#pragma unroll
  for (int k = 0; k < L; k++) m -= m / 2;
  return m;
}

// Components rooted at r = r0, r0 + rstride, ... < m_L, all in flight at
// once: slot j + 2^t holds the level-(L-1-t) partner of slot j (when it
// exists), so level k pairs slot j with slot j + 2^(L-1-k).
template <int L, typename T, bool KV, typename Mem, typename Isp>
__device__ __forceinline__ void msh_pass(T* A, uint64_t* Y, uint64_t m, uint64_t r0,
                                         uint64_t rstride, const Mem& mem, const Isp& isp) {
  constexpr int W = 1 << L;
  uint64_t mk[L], hk[L];
  uint64_t mm = m;
#pragma unroll
  for (int k = 0; k < L; k++) {
    mk[k] = mm;
    hk[k] = mm / 2;
    mm -= hk[k];
  }
  const uint64_t roots = mm;
  for (uint64_t r = r0; r < roots; r += rstride) {
    uint64_t x[W];
    uint32_t valid = 1;
    x[0] = r;
#pragma unroll
    for (int t = 0; t < L; t++) {
      const int k = L - 1 - t;
#pragma unroll
      for (int j = 0; j < (1 << t); j++) {
        const bool v = ((valid >> j) & 1u) && x[j] < hk[k];
        x[j + (1 << t)] = mk[k] - 1 - x[j];
        valid |= (uint32_t)v << (j + (1 << t));
      }
    }
    T key[W];
    uint64_t pos[W];
#pragma unroll
    for (int j = 0; j < W; j++) {
      pos[j] = mem(x[j]);
      if ((valid >> j) & 1u) key[j] = ldcg(&A[pos[j]]);
    }
    uint64_t src[KV ? W : 1];
    if constexpr (KV) {
#pragma unroll
      for (int j = 0; j < W; j++) src[j] = pos[j];
    }
    uint32_t changed = 0;
#pragma unroll
    for (int k = 0; k < L; k++) {
      const int t = L - 1 - k;
#pragma unroll
      for (int j = 0; j < (1 << t); j++) {
        const int q = j + (1 << t);
        if (((valid >> q) & 1u) && isp(key[j]) && !isp(key[q])) {
          const T u = key[j];
          key[j] = key[q];
          key[q] = u;
          changed |= (1u << j) | (1u << q);
          if constexpr (KV) {
            const uint64_t w = src[j];
            src[j] = src[q];
            src[q] = w;
          }
        }
      }
    }
    if (!changed) continue;
    if constexpr (KV) {
      uint64_t yv[W];
#pragma unroll
      for (int j = 0; j < W; j++)
        if ((changed >> j) & 1u) yv[j] = ldcg(&Y[src[j]]);
#pragma unroll
      for (int j = 0; j < W; j++)
        if ((changed >> j) & 1u) Y[pos[j]] = yv[j];
    }
#pragma unroll
    for (int j = 0; j < W; j++)
      if ((changed >> j) & 1u) A[pos[j]] = key[j];
  }
}

// ---- Values kept in the order of a block's keys (Sec. 3, Lemma bitstore2).
// L = bit length of the range size; the first 4L + 2 keys of a block (at
// logical position s) are 2L + 1 adjacent pairs.  The first write reorders
// the pairs, keeping their relative order, so that the kind making up at
// least half of them comes first: unequal pairs (at least L + 1) hold bit k
// of the value in the order of pair k < L (first > second <=> 1); otherwise
// the second key of equal pair k, 1 <= k <= L, is overwritten with bit k - 1.
// Pair 0 tells the kinds apart.  One warp per block; pair p = lane + 32 w.
constexpr uint32_t kMaxValueBits = 40;          // ranges below 2^40 keys
constexpr uint32_t kPairWords = (2 * kMaxValueBits + 1 + 31) / 32;

// The first write of v into the block at s.
template <typename T, typename Mem>
__device__ __forceinline__ void warp_value_first(T* A, uint64_t s, uint32_t L, uint64_t v,
                                                 const Mem& mem) {
  const uint32_t lane = threadIdx.x & 31u, P = 2 * L + 1, lt = (1u << lane) - 1u;
  T a[kPairWords], b[kPairWords];
  uint32_t uneq[kPairWords], inm[kPairWords], nuneq = 0;
#pragma unroll
  for (uint32_t w = 0; w < kPairWords; w++) {
    const uint32_t p = lane + 32 * w;
    if (p < P) {
      a[w] = ldcg(&A[mem(s + 2 * p)]);
      b[w] = ldcg(&A[mem(s + 2 * p + 1)]);
    }
    inm[w] = __ballot_sync(0xffffffffu, p < P);
    uneq[w] = __ballot_sync(0xffffffffu, p < P && a[w] != b[w]);
    nuneq += __popc(uneq[w]);
  }
  const bool order_kind = nuneq >= L + 1;
  uint32_t want[kPairWords], nwant = 0;
#pragma unroll
  for (uint32_t w = 0; w < kPairWords; w++) {
    want[w] = order_kind ? uneq[w] : (inm[w] & ~uneq[w]);
    nwant += __popc(want[w]);
  }
  uint32_t wb = 0, ub = 0;
#pragma unroll
  for (uint32_t w = 0; w < kPairWords; w++) {
    const uint32_t p = lane + 32 * w;
    const bool wanted = (want[w] >> lane) & 1u;
    const uint32_t unw = inm[w] & ~want[w];
    const uint32_t q = wanted ? wb + __popc(want[w] & lt) : nwant + ub + __popc(unw & lt);
    wb += __popc(want[w]);
    ub += __popc(unw);
    if (p < P) {
      T f = a[w], g = b[w];
      if (order_kind && q < L) {
        const bool bit = (v >> q) & 1u;
        const T lo = a[w] < b[w] ? a[w] : b[w], hi = a[w] < b[w] ? b[w] : a[w];
        f = bit ? hi : lo;
        g = bit ? lo : hi;
      } else if (!order_kind && q >= 1 && q <= L) {
        g = (T)((v >> (q - 1)) & 1u);
      }
      A[mem(s + 2 * q)] = f;  // every pair was read above, before any write
      A[mem(s + 2 * q + 1)] = g;
    }
  }
}

// Adds `off` to the value of the block at s (a later write: the kinds and
// the pair order stay).
template <typename T, typename Mem>
__device__ __forceinline__ void warp_value_add(T* A, uint64_t s, uint32_t L, uint64_t off,
                                               const Mem& mem) {
  const uint32_t lane = threadIdx.x & 31u;
  T a[2], b[2];
#pragma unroll
  for (uint32_t w = 0; w < 2; w++) {
    const uint32_t p = lane + 32 * w;
    if (p <= L) {
      a[w] = ldcg(&A[mem(s + 2 * p)]);
      b[w] = ldcg(&A[mem(s + 2 * p + 1)]);
    }
  }
  const bool order_kind = __shfl_sync(0xffffffffu, a[0], 0) != __shfl_sync(0xffffffffu, b[0], 0);
  uint64_t v = 0;
#pragma unroll
  for (uint32_t w = 0; w < 2; w++) {
    const uint32_t p = lane + 32 * w;
    const bool bit = order_kind ? (p < L && a[w] > b[w]) : (p >= 1 && p <= L && b[w] != (T)0);
    v |= (uint64_t)__ballot_sync(0xffffffffu, bit) << (32 * w);
  }
  if (!order_kind) v >>= 1;
  const uint64_t nv = v + off;
#pragma unroll
  for (uint32_t w = 0; w < 2; w++) {
    const uint32_t p = lane + 32 * w;
    if (order_kind && p < L) {
      const bool bit = (nv >> p) & 1u;
      if (bit != (a[w] > b[w])) {
        A[mem(s + 2 * p)] = b[w];
        A[mem(s + 2 * p + 1)] = a[w];
      }
    } else if (!order_kind && p >= 1 && p <= L) {
      const T g = (T)((nv >> (p - 1)) & 1u);
      if (g != b[w]) A[mem(s + 2 * p + 1)] = g;
    }
  }
}

// Puts back the keys the overwrite kind replaced in the block at s.
template <typename T, typename Mem>
__device__ __forceinline__ void warp_value_restore(T* A, uint64_t s, uint32_t L, const Mem& mem) {
  const uint32_t lane = threadIdx.x & 31u;
  const T a0 = ldcg(&A[mem(s)]), b0 = ldcg(&A[mem(s + 1)]);
  if (a0 != b0) return;  // the order kind moved keys only
#pragma unroll
  for (uint32_t w = 0; w < 2; w++) {
    const uint32_t p = lane + 32 * w;
    if (p >= 1 && p <= L) A[mem(s + 2 * p + 1)] = ldcg(&A[mem(s + 2 * p)]);
  }
}

template <typename T, bool KV, bool IMP>
__global__ void __launch_bounds__(kLT, 2) lowspace_kernel(T* keys, uint64_t* vals, LowArgs a,
                                                       TaskScratch S) {
  static_assert(!(IMP && KV), "values in key order: keys only");
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
    if (tid == 0) atomicOr(S.status, kStatTimeout | kSiteLowspace);
  };

  uint64_t lo = a.lo, hi = a.hi;
  if (a.range_desc) {
    lo = __ldcg(&a.range_desc->vmin);
    hi = __ldcg(&a.range_desc->vmax);
    if (lo >= hi) { lo = 0; hi = 0; }
  }
  const uint64_t n = hi - lo;
  // an empty range from a descriptor (nothing was handed over): every CTA
  // reads the same record, so all leave here together
  if (a.range_desc && n == 0) {
    if (leader && a.split) *a.split = 0;
    return;
  }
  T* A = keys + lo;
  uint64_t* Y = KV ? vals + lo : nullptr;
  const T pivot = (T)a.pivot;
  auto stamp = [&](int k) {
    if (leader) a.tl[k] = global_timer_ns();
  };
  stamp(0);

  // ---- 1. count, role swap
  {
    unsigned long long c =
        count_span(A, 0, n, gtid, gstride, [&](T x) { return x <= pivot; });
    c = cta_sum(c, red);
    if (tid == 0) __stcg(&a.cta[blockIdx.x], c);
  }
  if (!grid_barrier(S.bar, gridDim.x, &flag)) { fail(); return; }
  // every CTA adds up all CTAs' counts (the words are rewritten only after
  // the next grid barrier)
  unsigned long long cpart = 0;
  for (uint32_t c2 = tid; c2 < gridDim.x; c2 += kLT) cpart += __ldcg(&a.cta[c2]);
  const uint64_t cnt = cta_sum(cpart, red);
  if (leader && a.split) *a.split = cnt;
  stamp(1);
  if (n < 2) return;
  const bool flip = 2 * (n - cnt) < n;
  auto mem = [&](uint64_t i) -> uint64_t { return flip ? n - 1 - i : i; };
  auto isp = [&](T x) -> bool { return flip ? (x > pivot) : (x <= pivot); };


  // ---- 2. MakeSuccessorHeavy, kMshFuse levels per pass
  uint64_t m = n;
  while (m > 1) {
    const uint64_t mL = msh_after<kMshFuse<KV>>(m);
    if (m / 2 >= kMshSmall) {
      msh_pass<kMshFuse<KV>, T, KV>(A, Y, m, gtid, gstride, mem, isp);
      if (!grid_barrier(S.bar, gridDim.x, &flag)) { fail(); return; }
      m = mL;
    } else {
      if (blockIdx.x == 0) {
        while (m > 1) {
          msh_pass<kMshFuse<KV>, T, KV>(A, Y, m, tid, kLT, mem, isp);
          __syncthreads();
          m = msh_after<kMshFuse<KV>>(m);
        }
      }
      m = 1;
      if (!grid_barrier(S.bar, gridDim.x, &flag)) { fail(); return; }
    }
  }

  stamp(2);

  // ---- 3. block prefix: v[i] = predecessors in blocks 0..i (explicit), or
  // the predecessors before block i kept in the order of its keys
  const uint64_t B = a.B;
  const uint64_t nb = n / B;
  const uint32_t Lb = 64u - (uint32_t)__clzll((long long)n);  // bits of a value in [0, n]
  if constexpr (IMP) {
    if (Lb > kMaxValueBits || B < 4ull * Lb + 2) {  // the host checks this first
      if (tid == 0) atomicOr(S.status, kStatRing);
      return;
    }
    if (nb > 0) {
      // every CTA owns the blocks [b0, b1), every warp a contiguous run
      // [w0, w1) of them: the warp counts each block and writes into it the
      // count before it within the run; after one CTA barrier and one grid
      // barrier it adds the totals of the runs and CTAs before (a write of at
      // most L pairs per block)
      const uint64_t bpc = (nb + gridDim.x - 1) / gridDim.x;
      const uint64_t b0 = min((uint64_t)blockIdx.x * bpc, nb), b1 = min(b0 + bpc, nb);
      const uint64_t bpw = (b1 - b0 + kLT / 32 - 1) / (kLT / 32);
      const uint64_t w0 = min(b0 + warp * bpw, b1), w1 = min(w0 + bpw, b1);
      unsigned long long run = 0;
      for (uint64_t b = w0; b < w1; b++) {
        const uint64_t s0 = b * B, e = (b + 1 == nb) ? n : s0 + B;
        unsigned long long cw = flip ? count_span(A, n - e, n - s0, lane, 32, isp)
                                     : count_span(A, s0, e, lane, 32, isp);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cw += __shfl_xor_sync(0xffffffffu, cw, o);
        warp_value_first(A, s0, Lb, run, mem);
        run += cw;
      }
      __syncthreads();
      if (lane == 0) red[warp] = run;
      __syncthreads();
      unsigned long long before = 0, tot = 0;
      for (uint32_t w = 0; w < kLT / 32; w++) {
        const unsigned long long x = red[w];
        tot += x;
        if (w < warp) before += x;
      }
      if (tid == 0) __stcg(&a.cta[blockIdx.x], tot);
      if (!grid_barrier(S.bar, gridDim.x, &flag)) { fail(); return; }
      unsigned long long off = 0;
      for (uint32_t c2 = tid; c2 < blockIdx.x; c2 += kLT) off += __ldcg(&a.cta[c2]);
      off = cta_sum(off, red) + before;
      if (off != 0)
        for (uint64_t b = w0; b < w1; b++) warp_value_add(A, b * B, Lb, off, mem);
      if (!grid_barrier(S.bar, gridDim.x, &flag)) { fail(); return; }
    }
  } else {
    if (nb > a.nb_cap) {  // never expected: the host sizes the scratch for the array
      if (tid == 0) atomicOr(S.status, kStatRing);
      return;
    }
    if (nb > 0) {
      // every CTA owns the blocks [b0, b1); its warps count one block each
      // (16-byte loads) into v[b], the CTA turns those counts into an
      // inclusive prefix over its range, then adds the totals of the CTAs
      // before it
      const uint64_t bpc = (nb + gridDim.x - 1) / gridDim.x;
      const uint64_t b0 = min((uint64_t)blockIdx.x * bpc, nb), b1 = min(b0 + bpc, nb);
      unsigned long long* V = reinterpret_cast<unsigned long long*>(a.v);
      for (uint64_t b = b0 + warp; b < b1; b += kLT / 32) {
        const uint64_t s = b * B, e = (b + 1 == nb) ? n : s + B;
        const uint32_t c = flip ? count_span(A, n - e, n - s, lane, 32, isp)
                                : count_span(A, s, e, lane, 32, isp);
        unsigned long long cw = c;  // a block may hold more than 2^32 keys
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cw += __shfl_xor_sync(0xffffffffu, cw, o);
        if (lane == 0) __stcg(&V[b], cw);
      }
      __syncthreads();
      // thread tid sums the counts [c0, c1) of its share of the range
      const uint64_t per = (b1 - b0 + kLT - 1) / kLT;
      const uint64_t c0 = min(b0 + tid * per, b1), c1 = min(c0 + per, b1);
      unsigned long long own = 0;
      for (uint64_t b = c0; b < c1; b++) own += __ldcg(&V[b]);
      // exclusive scan of the shares across the CTA
      unsigned long long incl = own;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long w = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += w;
      }
      __syncthreads();
      if (lane == 31) red[warp] = incl;
      __syncthreads();
      unsigned long long before = incl - own;
      for (uint32_t w = 0; w < warp; w++) before += red[w];
      unsigned long long ctatot = 0;
      for (uint32_t w = 0; w < kLT / 32; w++) ctatot += red[w];
      if (tid == 0) __stcg(&a.cta[blockIdx.x], ctatot);
      if (!grid_barrier(S.bar, gridDim.x, &flag)) { fail(); return; }
      unsigned long long off = 0;
      for (uint32_t c2 = tid; c2 < blockIdx.x; c2 += kLT) off += __ldcg(&a.cta[c2]);
      off = cta_sum(off, red);
      unsigned long long run = off + before;
      for (uint64_t b = c0; b < c1; b++) {
        run += __ldcg(&V[b]);
        __stcg(&V[b], run);
      }
      if (!grid_barrier(S.bar, gridDim.x, &flag)) { fail(); return; }
    }
  }
  stamp(3);
  if (IMP && a.prefix_only) return;

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
  const uint64_t gwarp = ((uint64_t)blockIdx.x * kLT + tid) >> 5;
  const uint64_t nwarps = gstride >> 5;
  if constexpr (IMP) {
    // the innermost prefix's blocks get their overwritten keys back first
    for (uint64_t b = gwarp; b < mbase / B; b += nwarps) warp_value_restore(A, b * B, Lb, mem);
    if (!grid_barrier(S.bar, gridDim.x, &flag)) { fail(); return; }
  }
  {
    // the innermost prefix, partitioned on chip: in memory it is [0, mbase)
    // or, for the reversed view, [n - mbase, n) with the roles back in place
    const uint64_t off = flip ? n - mbase : 0;
    const uint64_t t = coop_finish<T, KV, kLT>(A + off, KV ? Y + off : nullptr, mbase, pivot,
                                               S, smem_raw, &flag);
    if (t == ~0ull) { fail(); return; }
    if (!grid_barrier(S.bar, gridDim.x, &flag)) { fail(); return; }
  }
  stamp(4);
  // Reorder level by level, outward; one warp per block, rounds of 32 * kRU
  // keys: every predecessor of block i goes to v[i-1] + its rank in the block
  // (a successor inside the successor-heavy prefix, which is partitioned
  // already).  Blocks and their targets are disjoint, so the next round's
  // keys (of this block or the warp's next one) load while this round's
  // targets do.
  constexpr uint32_t kRU = KV ? 4 : (sizeof(T) == 4 ? 2 * kUnroll : kUnroll);
  static_assert(IMP ? 32 * kRU >= 2 * (kMaxValueBits + 1) : true, "a block's value in one round");
  // Explicit counters: a block's targets are one contiguous range starting
  // at v[i-1] and ending at v[i], so a round's targets lie in the window
  // [y, y + 32 kWR) -- known once the round before has been ranked.  That
  // window (keys, and with payloads their values) is loaded with the round's
  // keys (and with payloads the round's own values), a round ahead, up to the
  // block's last target, and staged in the warp's shared memory (free during
  // this phase), so no round waits on its target loads.  Targets are disjoint
  // from the sources and from other blocks' targets, so reading them a round
  // early is safe.  4-byte keys take rounds of twice the keys and a window of
  // 10 rows (320 keys): the view's predecessors are at most half the keys, so
  // a round's targets nearly always fit; a target past the window is loaded
  // directly.
  constexpr bool kWin = !IMP;
  constexpr uint32_t kWR = sizeof(T) == 4 ? 10 : kRU;  // window rows
  static_assert(kWR <= kRU, "a window of at most a round");
  static_assert(!kWin || (kLT / 32) * 32 * kWR * (sizeof(T) + (KV ? 8 : 0)) <=
                             level_smem_bytes<T, KV>(),
                "the target windows fit the dynamic shared memory");
  T* const tw = reinterpret_cast<T*>(smem_raw) +
                (size_t)warp * (32 * kWR) * (KV ? 2 * sizeof(uint64_t) / sizeof(T) : 1);
  uint64_t* const twv = reinterpret_cast<uint64_t*>(tw + 32 * kWR);  // values (payloads only)
  const uint32_t lt = (1u << lane) - 1u;
  const unsigned long long* V = reinterpret_cast<const unsigned long long*>(a.v);
  for (int j = L - 1; j >= 0; j--) {
    const uint64_t M = levM[j], t0 = levT[j], NB = levNB[j];
    uint64_t i = t0 + gwarp;
    if (i < NB) {
      uint64_t r0 = i * B, e = (i + 1 == NB) ? M : r0 + B;
      uint64_t y = IMP ? 0 : __ldcg(&V[i - 1]);  // kept in key order: read below
      // the end of the block's targets (window loads stop there: at a 1% or
      // 99% pivot a round has a few targets, not 32 kRU)
      uint64_t te = kWin ? __ldcg(&V[i]) : 0;
      T x[kRU];
      T w[kWin ? kWR : 1];  // the round's target window, lane l holding y + 32 u + l
      constexpr bool kWV = kWin && KV;
      uint64_t xv[kWV ? kRU : 1], wv[kWV ? kWR : 1];  // the round's values, the window's
#pragma unroll
      for (uint32_t u = 0; u < kRU; u++) {
        const uint64_t q = r0 + 32ull * u + lane;
        if (q < e) {
          x[u] = ldcg(&A[mem(q)]);
          if constexpr (kWV) xv[u] = ldcg(&Y[mem(q)]);
        }
        if constexpr (kWin) {
          const uint64_t qt = y + 32ull * u + lane;
          if (u < kWR && qt < te) {
            w[u] = ldcg(&A[mem(qt)]);
            if constexpr (kWV) wv[u] = ldcg(&Y[mem(qt)]);
          }
        }
      }
      for (;;) {
        // the next round: the rest of this block, else the warp's next block
        uint64_t i1 = i, r1 = r0 + 32ull * kRU, e1 = e;
        const bool next_block = r1 >= e;
        if (next_block) {
          i1 = i + nwarps;
          r1 = i1 * B;
          e1 = (i1 + 1 == NB) ? M : r1 + B;
        }
        const bool more = i1 < NB;
        if constexpr (IMP) {
          if (r0 == i * B) {  // the block's first round holds its value
            // pair p is lanes 2p, 2p + 1 (mod 32) of round word p / 16
            constexpr uint32_t kDecU = (kMaxValueBits + 1 + 15) / 16;
            T nbv[kDecU];
#pragma unroll
            for (uint32_t u = 0; u < kDecU; u++) nbv[u] = __shfl_down_sync(0xffffffffu, x[u], 1);
            const bool order_kind =
                __shfl_sync(0xffffffffu, x[0], 0) != __shfl_sync(0xffffffffu, nbv[0], 0);
            const bool even = (lane & 1u) == 0;
            uint64_t val = 0;
#pragma unroll
            for (uint32_t u = 0; u < kDecU; u++) {
              const uint32_t p = 16 * u + (lane >> 1);
              const bool bit = even && (order_kind ? (p < Lb && x[u] > nbv[u])
                                                   : (p >= 1 && p <= Lb && nbv[u] != (T)0));
              const uint32_t bm = __ballot_sync(0xffffffffu, bit);
              uint32_t c = 0;
#pragma unroll
              for (uint32_t j = 0; j < 16; j++) c |= ((bm >> (2 * j)) & 1u) << j;
              val |= (uint64_t)c << (16 * u);
            }
            if (!order_kind) {
              val >>= 1;
#pragma unroll
              for (uint32_t u = 0; u < kDecU; u++) {
                const T ev = __shfl_up_sync(0xffffffffu, x[u], 1);
                const uint32_t p = 16 * u + (lane >> 1);
                if (!even && p >= 1 && p <= Lb) {
                  x[u] = ev;
                  A[mem(r0 + 32ull * u + lane)] = ev;
                }
              }
            }
            y = val;
          }
        }
        if constexpr (kWin) {  // the round's target window into shared memory
          __syncwarp();
#pragma unroll
          for (uint32_t u = 0; u < kWR; u++) {
            tw[32 * u + lane] = w[u];
            if constexpr (kWV) twv[32 * u + lane] = wv[u];
          }
          __syncwarp();
        }
        uint32_t f = 0;
#pragma unroll
        for (uint32_t u = 0; u < kRU; u++)
          f |= (r0 + 32ull * u + lane < e && isp(x[u]) ? 1u : 0u) << u;
        T z[kRU];
        uint32_t tg[kRU];  // target offsets from y
        uint64_t py[KV ? kRU : 1], pz[KV ? kRU : 1];
        uint32_t run = 0;
#pragma unroll
        for (uint32_t u = 0; u < kRU; u++) {
          const uint32_t bal = __ballot_sync(0xffffffffu, (f >> u) & 1u);
          tg[u] = run + __popc(bal & lt);
          if ((f >> u) & 1u) {
            if constexpr (kWin) {
              if (kWR == kRU || tg[u] < 32 * kWR) {
                z[u] = tw[tg[u]];
              } else {  // past the window (4-byte keys, rare): load it here
                z[u] = ldcg(&A[mem(y + tg[u])]);
              }
              if constexpr (kWV) {
                pz[u] = twv[tg[u]];
                py[u] = xv[u];
              }
            } else {
              const uint64_t pt = mem(y + tg[u]);
              z[u] = ldcg(&A[pt]);
              if constexpr (KV) {
                pz[u] = ldcg(&Y[pt]);
                py[u] = ldcg(&Y[mem(r0 + 32ull * u + lane)]);
              }
            }
          }
          run += __popc(bal);
        }
        T xn[kRU];
        uint64_t xvn[kWV ? kRU : 1];
        uint64_t yn = y + run;
        if (more) {
          if (next_block) {
            yn = IMP ? 0 : __ldcg(&V[i1 - 1]);
            if constexpr (kWin) te = __ldcg(&V[i1]);
          }
#pragma unroll
          for (uint32_t u = 0; u < kRU; u++) {
            const uint64_t q = r1 + 32ull * u + lane;
            if (q < e1) {
              xn[u] = ldcg(&A[mem(q)]);
              if constexpr (kWV) xvn[u] = ldcg(&Y[mem(q)]);
            }
            if constexpr (kWin) {  // the next round's targets start at yn
              const uint64_t qt = yn + 32ull * u + lane;
              if (u < kWR && qt < te) {
                w[u] = ldcg(&A[mem(qt)]);
                if constexpr (kWV) wv[u] = ldcg(&Y[mem(qt)]);
              }
            }
          }
        }
#pragma unroll
        for (uint32_t u = 0; u < kRU; u++) {
          if ((f >> u) & 1u) {
            const uint64_t pt = mem(y + tg[u]), ps = mem(r0 + 32ull * u + lane);
            A[pt] = x[u];
            A[ps] = z[u];
            if constexpr (KV) {
              Y[pt] = py[u];
              Y[ps] = pz[u];
            }
          }
        }
        if (!more) break;
#pragma unroll
        for (uint32_t u = 0; u < kRU; u++) {
          x[u] = xn[u];
          if constexpr (kWV) xv[u] = xvn[u];
        }
        i = i1;
        r0 = r1;
        e = e1;
        y = yn;
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

namespace {

template <typename T, bool KV, bool IMP>
cudaError_t launch_lowspace_impl(T* keys, uint64_t* vals, uint64_t lo, uint64_t hi,
                                 uint64_t n_cap, const LevelDesc* range_desc, T pivot, uint64_t B,
                                 uint64_t base_keys, int prefix_only, void* var,
                                 const TaskScratch& S, uint64_t* split, LaunchCfg& cfg) {
  cudaStream_t st = cfg.stream;
  // the scratch is laid out for the largest range it may see (the range may
  // only be known on the device); values kept in key order need no counters
  const uint64_t nb = (B && !IMP) ? n_cap / B : 0;
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
  a.tl = reinterpret_cast<unsigned long long*>(p + 256);
  a.split = split;
  a.prefix_only = prefix_only;
  const size_t smem = level_smem_bytes<T, KV>();
  cudaError_t e = cudaFuncSetAttribute(lowspace_kernel<T, KV, IMP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // a cooperative grid must fit on the device at once: size it by this kernel
  int dev = 0, sms = 0, per = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, lowspace_kernel<T, KV, IMP>, kLT,
                                                         smem)) != cudaSuccess)
    return e;
  uint32_t grid = cfg.grid;
  if ((uint64_t)sms * (uint64_t)(per < 1 ? 1 : per) < grid) grid = (uint32_t)(sms * (per < 1 ? 1 : per));
  const uint64_t cap = (uint64_t)grid * Coop<T, KV>::Keys;
  a.base_keys = base_keys < cap ? base_keys : cap;
  if (a.base_keys < 5 * B) a.base_keys = 0;  // the paper's base case decides
  if (cfg.phase_stamps) {  // the caller reads the phase timestamps: no stale ones
    e = cudaMemsetAsync(a.tl, 0, 8 * kLowPhases, st);
    if (e != cudaSuccess) return e;
    *cfg.phase_stamps = a.tl;
  }
  e = launch_cooperative(lowspace_kernel<T, KV, IMP>, grid, kLT, smem, st, keys, vals, a, S);
  cfg.launches++;
  return e;
}

}  // namespace

template <typename T, bool KV>
cudaError_t launch_lowspace(T* keys, uint64_t* vals, uint64_t lo, uint64_t hi, uint64_t n_cap,
                            const LevelDesc* range_desc, T pivot, uint64_t B, uint64_t base_keys,
                            void* var, const TaskScratch& S, uint64_t* split, LaunchCfg& cfg) {
  return launch_lowspace_impl<T, KV, false>(keys, vals, lo, hi, n_cap, range_desc, pivot, B,
                                            base_keys, 0, var, S, split, cfg);
}

size_t lowspace_implicit_scratch_bytes(uint32_t grid) { return lowspace_scratch_bytes(0, 1, grid); }

uint32_t lowspace_value_bits(uint64_t n) {
  uint32_t L = 0;
  while (L < 64 && (n >> L) != 0) L++;
  return L;
}

uint32_t lowspace_value_bits_max() { return kMaxValueBits; }

template <typename T>
cudaError_t launch_lowspace_implicit(T* keys, uint64_t n, T pivot, uint64_t B,
                                     uint64_t base_keys, int prefix_only, void* var,
                                     const TaskScratch& S, uint64_t* split, LaunchCfg& cfg) {
  return launch_lowspace_impl<T, false, true>(keys, nullptr, 0, n, n, nullptr, pivot, B,
                                              base_keys, prefix_only, var, S, split, cfg);
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

template cudaError_t launch_lowspace_implicit<uint64_t>(uint64_t*, uint64_t, uint64_t, uint64_t,
                                                        uint64_t, int, void*, const TaskScratch&,
                                                        uint64_t*, LaunchCfg&);
template cudaError_t launch_lowspace_implicit<uint32_t>(uint32_t*, uint64_t, uint32_t, uint64_t,
                                                        uint64_t, int, void*, const TaskScratch&,
                                                        uint64_t*, LaunchCfg&);

}  // namespace lp
