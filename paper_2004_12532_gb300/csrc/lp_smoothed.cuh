// lp_smoothed.cuh -- the Smoothed Striding partial partition step on sm_103a
// (Sec. 4 of arXiv 2004.12532, "Formal Algorithm Description" and the figure
// "Smoothed Striding Algorithm").
//
// GPU mapping.  Each warp owns one group U_i at a time (the paper partitions
// every U_i serially, one processor per group).  The group's lines -- line
// j*g + (X[j]+i) mod g of every chunk j -- form a sequence of nl lines in
// group order, which the warp partitions in place with the paper's serial
// two-pointer scan taken one line at a time:
//   * the warp holds the lowest unfinished line L and the highest unfinished
//     line R in registers (lane l holds vectors l and 32+l of each);
//   * the j-th successor of L and the j-th predecessor of R are swapped for
//     j < min(#successors(L), #predecessors(R)) -- ranks (lane by lane)
//     come from one warp scan of per-lane counts, the keys cross through a
//     small shared-memory buffer;
//   * whichever line became pure (L all predecessors, R all successors) is
//     written straight back with coalesced 16-byte stores, and the next line
//     of that side is taken; the last line left is partitioned on its own;
//   * lane 0 keeps Q lines per side in flight with 1-D bulk asynchronous
//     copies (TMA) into shared-memory stages, each completing on an mbarrier.
// Every line is read once and written once: one read and one write of every
// key, the I/O of the paper's Prop. 4.2.  The group ends predecessors first in
// its own slot order, as the paper's serial partition leaves it, so k_i and
// v_i are the paper's.
//
// The random offsets X[j] are computed 32 at a time, one per lane, and
// fetched by shuffle.  v_min / v_max are reduced with 64-bit atomic min / max
// into the level descriptor (order-independent, deterministic).  There are no
// CTA-wide barriers on this path: warps run independently.
#pragma once
#include "lp_device.cuh"
#include "lp_plan.h"

namespace lp {

// One record per level of one partition task, in device memory.
struct LevelDesc {
  unsigned long long vmin;   // min over groups of v_i (absolute position)
  unsigned long long vmax;   // max over groups of v_i
  unsigned long long count;  // sum over groups of k_i
  unsigned long long lo, hi; // the (aligned) range this level worked on
  unsigned long long b, g;   // parameters used (g == 0: the on-chip base case)
  unsigned long long t_start;  // device time (ns) when the level started
};

// Arguments of one level launch.
struct LevelArgs {
  uint64_t lo, hi;           // range when `in` is null
  uint64_t body_lo, body_hi; // 16-byte aligned body of the array
  uint64_t pivot;
  uint64_t seed;
  uint64_t level;
  uint64_t fixed_b, fixed_g; // nonzero: use these parameters
  int strided;               // X == 0
  int force_finish;          // the last level: finish whatever is left
};

template <typename T, bool KV>
struct Tr {
  static constexpr uint32_t K = sizeof(T);
  // key bytes per line, max; Q lines in flight per side
  static constexpr uint32_t LineBytes = max_line_bytes(sizeof(T));
  static constexpr uint32_t Q = LineBytes == 2048u ? 2u : 4u;
  static constexpr uint32_t Stages = 2u * Q;
  static constexpr uint32_t LineKeys = LineBytes / K;
  static constexpr uint32_t V = 16u / K;                        // keys per 16-byte vector
  static constexpr uint32_t A = 16u / K;                        // alignment unit in keys
  static constexpr uint32_t VPL = LineBytes / 16u / 32u;        // vectors per lane per line
  static constexpr uint32_t Warps = KV ? 4u : 8u;               // groups in flight per CTA
  static constexpr uint32_t Threads = 32u * Warps;
  // one CTA partitions ranges up to this many keys in shared memory
  static constexpr uint32_t FinishKeys = kFinishBytes / (K + (KV ? 8u : 0u));
};

template <typename T, bool KV>
struct __align__(128) WarpSmem {
  static constexpr uint32_t S = Tr<T, KV>::Stages;
  T stage[S][Tr<T, KV>::LineKeys];
  T xbuf[2][Tr<T, KV>::LineKeys];
  uint64_t vstage[KV ? S : 1][KV ? Tr<T, KV>::LineKeys : 2];
  uint64_t vxbuf[KV ? 2 : 1][KV ? Tr<T, KV>::LineKeys : 2];
  uint64_t bar[S];
  uint32_t st_line[S];   // line (within the range) loaded into each stage
  uint32_t st_len[S];    // ... and its length in keys
};

template <typename T, bool KV>
constexpr size_t level_smem_bytes() {
  constexpr size_t w = sizeof(WarpSmem<T, KV>) * Tr<T, KV>::Warps;
  constexpr size_t f = (size_t)Tr<T, KV>::FinishKeys * (sizeof(T) + (KV ? 8 : 0)) + 256;
  return w > f ? w : f;
}

template <typename T>
__device__ __forceinline__ void load_vec(const T* p, T (&x)[16 / sizeof(T)]) {
  if constexpr (sizeof(T) == 8) {
    ulonglong2 v = *reinterpret_cast<const ulonglong2*>(p);
    x[0] = v.x; x[1] = v.y;
  } else {
    uint4 v = *reinterpret_cast<const uint4*>(p);
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
  }
}

template <typename T>
__device__ __forceinline__ void store_vec(T* p, const T (&x)[16 / sizeof(T)]) {
  if constexpr (sizeof(T) == 8) {
    *reinterpret_cast<ulonglong2*>(p) = make_ulonglong2(x[0], x[1]);
  } else {
    *reinterpret_cast<uint4*>(p) = make_uint4(x[0], x[1], x[2], x[3]);
  }
}

// One line of a group in registers: lane l holds vectors u*32 + l, u < VPL.
template <typename T, bool KV>
struct LineReg {
  T x[Tr<T, KV>::VPL][Tr<T, KV>::V];
  uint64_t y[KV ? Tr<T, KV>::VPL : 1][KV ? Tr<T, KV>::V : 1];
  uint32_t pred;   // bit u*V+v: key (u, v) is a predecessor
  uint32_t keys;   // bit u*V+v: key (u, v) exists (vector u*32 + lane is in the line)
  uint32_t gl;     // line index within the range (warp-uniform)
  uint32_t len;    // keys in the line (warp-uniform)
};

// Partition group i of step G over the range starting at `base` (`vbase`
// for payloads).  Called by all 32 lanes of one warp with the same arguments;
// control is warp-uniform, lane 0 issues the bulk copies.  `phase` holds one
// parity bit per stage and persists across the warp's groups.  Returns false
// if a bounded wait gave up (after draining the warp's copies in flight);
// k receives the group's predecessor count.  Lines are indexed in 32 bits
// (the range has fewer than 2^31 lines; the host and parameter rule keep it so).
template <typename T, bool KV>
__device__ bool warp_pair_group(T* __restrict__ base, uint64_t* __restrict__ vbase,
                                const StepGeom& G, uint32_t i, int32_t nl, T pivot,
                                WarpSmem<T, KV>& sm, uint32_t& phase, uint64_t& k,
                                uint32_t* status) {
  using R = Tr<T, KV>;
  constexpr uint32_t V = R::V, VPL = R::VPL, NB = VPL * V;
  constexpr uint32_t FULL = 0xffffffffu;
  static_assert(NB < 32, "slot masks of 32-bit words");
  constexpr uint32_t kAllSlots = (1u << NB) - 1u;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t lt = (1u << lane) - 1u;
  k = 0;
  if (nl <= 0) return true;
  uint32_t kl = 0;  // this lane's predecessors (the group's k is their sum)

  // per-step constants in 32 bits
  const uint32_t g32 = (uint32_t)G.g, b32 = (uint32_t)G.b;
  const uint32_t last_line = (uint32_t)(G.L - 1);
  const uint32_t last_len = (uint32_t)(G.n - (G.L - 1) * G.b);

  // X windows: lane l holds X[wf + l] (front) and X[wb - l] (back)
  int32_t wf = -64, wb = -64;
  uint32_t xf = 0, xb = 0;

  PairCtl c;
  pair_init(c, nl);

  auto issue = [&](int32_t line, uint32_t st, bool front) {
    uint32_t x = 0;
    if (!G.strided) {
      if (front) {
        if (line < wf || line >= wf + 32) {
          wf = line;
          const uint64_t j = (uint64_t)(uint32_t)wf + lane;
          xf = j < G.s ? (uint32_t)range_of(sm_stream(G.sigma, j), G.g) : 0u;
        }
        x = __shfl_sync(FULL, xf, line - wf);
      } else {
        if (line > wb || line <= wb - 32) {
          wb = line;
          const int32_t j = wb - (int32_t)lane;
          xb = j >= 0 ? (uint32_t)range_of(sm_stream(G.sigma, (uint64_t)j), G.g) : 0u;
        }
        x = __shfl_sync(FULL, xb, wb - line);
      }
    }
    uint32_t off = x + i;
    if (off >= g32) off -= g32;
    const uint32_t gl = (uint32_t)line * g32 + off;
    if (lane == 0) {
      const uint32_t len = gl == last_line ? last_len : b32;
      sm.st_line[st] = gl;
      sm.st_len[st] = len;
      const uint32_t bytes = len * R::K;
      mbar_arrive_expect_tx(&sm.bar[st], KV ? 2u * bytes : bytes);
      bulk_load(&sm.stage[st][0], base + (size_t)gl * b32, bytes, &sm.bar[st]);
      if constexpr (KV) bulk_load(&sm.vstage[st][0], vbase + (size_t)gl * b32, bytes, &sm.bar[st]);
    }
  };
  // take an issued line into registers; refill its stage; false on timeout
  auto take = [&](int32_t line, LineReg<T, KV>& Lr) -> bool {
    const uint32_t st = pair_stage_of<R::Q>(c, line);
    const bool arrived = mbar_wait_bounded(&sm.bar[st], (phase >> st) & 1u);
    if (!__all_sync(FULL, arrived)) return false;
    phase ^= 1u << st;
    Lr.gl = sm.st_line[st];
    Lr.len = sm.st_len[st];
    const uint32_t nvec = Lr.len / V;
    uint32_t pred = 0, keys = 0;
    auto load_vector = [&](uint32_t u) {
      const uint32_t vec = u * 32u + lane;
      load_vec<T>(&sm.stage[st][vec * V], Lr.x[u]);
      if constexpr (KV) {
        const ulonglong2 w = *reinterpret_cast<const ulonglong2*>(&sm.vstage[st][vec * V]);
        Lr.y[u][0] = w.x; Lr.y[u][1] = w.y;
      }
#pragma unroll
      for (uint32_t v = 0; v < V; v++)
        if (Lr.x[u][v] <= pivot) pred |= 1u << (u * V + v);
    };
    if (NB > 8 && Lr.len == R::LineKeys) {  // a full line (warp-uniform; 4-byte keys,
                                            // ALU-bound): every vector exists
#pragma unroll
      for (uint32_t u = 0; u < VPL; u++) load_vector(u);
      keys = kAllSlots;
    } else {
#pragma unroll
      for (uint32_t u = 0; u < VPL; u++) {
        if (u * 32u + lane < nvec) {
          load_vector(u);
          keys |= ((1u << V) - 1u) << (u * V);
        }
      }
    }
    Lr.pred = pred;
    Lr.keys = keys;
    kl += __popc(pred);
    __syncwarp();  // every lane has read the stage: it may be refilled
    if (pair_can_issue(c)) {
      if (st < R::Q) { issue(c.fi, pair_stage_front<R::Q>(c.fi), true); c.fi++; }
      else { issue(c.bi, pair_stage_back<R::Q>(c, c.bi), false); c.bi--; }
    }
    return true;
  };
  auto store_line = [&](const LineReg<T, KV>& Lr) {
    T* dst = base + (size_t)Lr.gl * b32;
    auto store_vector = [&](uint32_t u) {
      const uint32_t vec = u * 32u + lane;
      store_vec<T>(dst + vec * V, Lr.x[u]);
      if constexpr (KV) {
        *reinterpret_cast<ulonglong2*>(vbase + (size_t)Lr.gl * b32 + vec * V) =
            make_ulonglong2(Lr.y[u][0], Lr.y[u][1]);
      }
    };
    if (NB > 8 && Lr.len == R::LineKeys) {  // a full line (warp-uniform; 4-byte keys)
#pragma unroll
      for (uint32_t u = 0; u < VPL; u++) store_vector(u);
    } else {
#pragma unroll
      for (uint32_t u = 0; u < VPL; u++)
        if ((Lr.keys >> (u * V)) & 1u) store_vector(u);
    }
  };

  for (uint32_t q = 0; q < R::Q; q++) {
    if (pair_can_issue(c)) { issue(c.fi, pair_stage_front<R::Q>(c.fi), true); c.fi++; }
    if (pair_can_issue(c)) { issue(c.bi, pair_stage_back<R::Q>(c, c.bi), false); c.bi--; }
  }
  __syncwarp();

  LineReg<T, KV> Lr, Rr;
  bool hasL = false, hasR = false, ok = true;
  for (;;) {
    if (!hasL && pair_has_unread(c)) {
      if (!take(c.fnext, Lr)) { ok = false; break; }
      c.fnext++;
      hasL = true;
    }
    if (!hasR && pair_has_unread(c)) {
      if (!take(c.bnext, Rr)) { ok = false; break; }
      c.bnext--;
      hasR = true;
    }
    if (!(hasL && hasR)) break;

    // swap the j-th successor of L with the j-th predecessor of R, both
    // numbered lane by lane (slots in order within a lane): one warp scan of
    // the per-lane counts, packed (successors of L low, predecessors of R high)
    const uint32_t lsucc = ~Lr.pred & Lr.keys;
    const uint32_t rpred = Rr.pred;
    const uint32_t own = (uint32_t)__popc(lsucc) | ((uint32_t)__popc(rpred) << 16);
    uint32_t incl = own;
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t tot = __shfl_sync(FULL, incl, 31);
    const uint32_t SL = tot & 0xffffu, PR = tot >> 16;
    const uint32_t m = min(SL, PR);
    if (m > 0) {
      const uint32_t exl = (incl - own) & 0xffffu, exr = (incl - own) >> 16;
      if constexpr (NB > 8) {
        // 16 slots per lane (4-byte keys: the slot work, not HBM, bounds
        // them).  Every wrong key of both lines goes to the exchange buffer
        // at its rank (successors of L from exl on, predecessors of R from exr
        // on, in slot order); only ranks below m are read back.  m =
        // min(SL, PR), so the wrong keys of the side with fewer all move and
        // the other side's movers are its lowest m ranks -- in each lane the
        // lowest of its wrong keys, cut in the one lane where rank m falls.
        // A pointer walks the buffer per side, stepping under the slot's own
        // predicate together with its store or load.
        static_assert(!KV, "key + payload lines hold 8 slots per lane");
        T* pl = &sm.xbuf[0][exl];
        T* pr = &sm.xbuf[1][exr];
#pragma unroll
        for (uint32_t j = 0; j < NB; j++) {
          const uint32_t u = j / V, v = j % V;
          if ((lsucc >> j) & 1u) *pl++ = Lr.x[u][v];
          if ((rpred >> j) & 1u) *pr++ = Rr.x[u][v];
        }
        // the movers: all wrong keys of the side with fewer, the first m of the other
        auto first_m = [&](uint32_t wrong, uint32_t ex) -> uint32_t {
          const uint32_t have = (uint32_t)__popc(wrong);
          if (ex >= m) return 0u;
          if (ex + have <= m) return wrong;
          uint32_t t = wrong;  // the lane holding rank m: keep its lowest m - ex
          for (uint32_t c = m - ex; c > 0; c--) t &= t - 1u;
          return wrong ^ t;
        };
        const uint32_t ml = SL <= PR ? lsucc : first_m(lsucc, exl);
        const uint32_t mr = PR <= SL ? rpred : first_m(rpred, exr);
        __syncwarp();
        // each side reads the other's keys at its own ranks
        const T* ql = &sm.xbuf[1][exl];
        const T* qr = &sm.xbuf[0][exr];
#pragma unroll
        for (uint32_t j = 0; j < NB; j++) {
          const uint32_t u = j / V, v = j % V;
          if ((ml >> j) & 1u) Lr.x[u][v] = *ql++;
          if ((mr >> j) & 1u) Rr.x[u][v] = *qr++;
        }
        Lr.pred |= ml;
        Rr.pred &= ~mr;
      } else {
        // 8 slots per lane: each slot's rank from a population count
        uint32_t rl[NB], rr[NB];
#pragma unroll
        for (uint32_t j = 0; j < NB; j++) {
          const uint32_t u = j / V, v = j % V;
          const uint32_t below = (1u << j) - 1u;
          rl[j] = ((lsucc >> j) & 1u) ? exl + __popc(lsucc & below) : 0xffffffffu;
          rr[j] = ((rpred >> j) & 1u) ? exr + __popc(rpred & below) : 0xffffffffu;
          if (rl[j] < m) {
            sm.xbuf[0][rl[j]] = Lr.x[u][v];
            if constexpr (KV) sm.vxbuf[0][rl[j]] = Lr.y[u][v];
          }
          if (rr[j] < m) {
            sm.xbuf[1][rr[j]] = Rr.x[u][v];
            if constexpr (KV) sm.vxbuf[1][rr[j]] = Rr.y[u][v];
          }
        }
        __syncwarp();
#pragma unroll
        for (uint32_t j = 0; j < NB; j++) {
          const uint32_t u = j / V, v = j % V;
          if (rl[j] < m) {
            Lr.x[u][v] = sm.xbuf[1][rl[j]];
            if constexpr (KV) Lr.y[u][v] = sm.vxbuf[1][rl[j]];
            Lr.pred |= 1u << j;
          }
          if (rr[j] < m) {
            Rr.x[u][v] = sm.xbuf[0][rr[j]];
            if constexpr (KV) Rr.y[u][v] = sm.vxbuf[0][rr[j]];
            Rr.pred &= ~(1u << j);
          }
        }
      }
      __syncwarp();  // the buffer is free for the next swap
    }
    if (SL <= PR) { store_line(Lr); hasL = false; }
    if (PR <= SL) { store_line(Rr); hasR = false; }
  }

  if (!ok) {
    // drain this warp's loads still in flight with bounded waits; the array
    // is left in an unspecified state and the status word says why
    if (lane == 0) {
      atomicOr(status, kStatTimeout | kSiteLine);
      for (int32_t l = c.fnext; l <= c.bnext; l++) {
        if (l >= c.fi && l <= c.bi) continue;  // never issued
        const uint32_t s2 = pair_stage_of<R::Q>(c, l);
        mbar_wait_bounded(&sm.bar[s2], (phase >> s2) & 1u);
      }
    }
    __syncwarp();
    return false;
  }

  // the one line left in hand: predecessors first, then successors
  if (hasL || hasR) {
    LineReg<T, KV>& F = hasL ? Lr : Rr;
    uint32_t bp[NB];
    uint32_t P = 0;
#pragma unroll
    for (uint32_t j = 0; j < NB; j++) {
      bp[j] = __ballot_sync(FULL, (F.pred >> j) & 1u);
      P += __popc(bp[j]);
    }
    uint32_t ap = 0, as = 0;
    T* dst = base + (size_t)F.gl * b32;
    uint64_t* vdst = KV ? vbase + (size_t)F.gl * b32 : nullptr;
#pragma unroll
    for (uint32_t j = 0; j < NB; j++) {
      const uint32_t u = j / V, v = j % V;
      const uint32_t bs = __ballot_sync(FULL, ((F.keys >> j) & 1u) && !((F.pred >> j) & 1u));
      if ((bp[j] >> lane) & 1u) {
        const uint32_t pos = ap + __popc(bp[j] & lt);
        dst[pos] = F.x[u][v];
        if constexpr (KV) vdst[pos] = F.y[u][v];
      } else if ((bs >> lane) & 1u) {
        const uint32_t pos = P + as + __popc(bs & lt);
        dst[pos] = F.x[u][v];
        if constexpr (KV) vdst[pos] = F.y[u][v];
      }
      ap += __popc(bp[j]);
      as += __popc(bs);
    }
  }
  k = __reduce_add_sync(FULL, kl);
  return true;
}

// Whole partition of a range of n <= FinishKeys keys by one CTA: keys staged
// in shared memory, each thread ranks a contiguous slice, and every key is
// written once to its final place (predecessors in order, then successors).
// Any alignment.  Called by all threads of the CTA.  Returns the count.
template <typename T, bool KV>
__device__ uint32_t cta_partition_smem(T* __restrict__ keys, uint64_t* __restrict__ vals,
                                       uint32_t n, T pivot, unsigned char* smem) {
  constexpr uint32_t NT = Tr<T, KV>::Threads;
  uint32_t* wsum = reinterpret_cast<uint32_t*>(smem);  // NT/32 <= 32 words
  T* sk = reinterpret_cast<T*>(smem + 128);
  uint64_t* sv = reinterpret_cast<uint64_t*>(
      smem + 128 + (((size_t)n * sizeof(T) + 15) & ~size_t(15)));
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  // through L2 (other CTAs may have written these), 8 loads in flight per thread
  constexpr uint32_t U = 8;
  for (uint32_t q0 = tid; q0 < n; q0 += NT * U) {
    T x[U];
    uint64_t y[KV ? U : 1];
#pragma unroll
    for (uint32_t u = 0; u < U; u++) {
      const uint32_t q = q0 + u * NT;
      if (q < n) {
        if constexpr (sizeof(T) == 8)
          x[u] = (T)__ldcg(reinterpret_cast<const unsigned long long*>(keys + q));
        else
          x[u] = (T)__ldcg(reinterpret_cast<const unsigned int*>(keys + q));
        if constexpr (KV) y[u] = __ldcg(reinterpret_cast<const unsigned long long*>(vals + q));
      }
    }
#pragma unroll
    for (uint32_t u = 0; u < U; u++) {
      const uint32_t q = q0 + u * NT;
      if (q < n) {
        sk[q] = x[u];
        if constexpr (KV) sv[q] = y[u];
      }
    }
  }
  __syncthreads();
  const uint32_t per = (n + NT - 1) / NT;
  const uint32_t s0 = min(n, tid * per), s1 = min(n, s0 + per);
  uint32_t cnt = 0;
  for (uint32_t q = s0; q < s1; q++) cnt += sk[q] <= pivot;
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
  uint32_t pp = wb + incl - cnt;
  uint32_t sp = tot + (s0 - pp);
  for (uint32_t q = s0; q < s1; q++) {
    const T x = sk[q];
    const uint32_t d = x <= pivot ? pp++ : sp++;
    keys[d] = x;
    if constexpr (KV) vals[d] = sv[q];
  }
  __syncthreads();
  return tot;
}

// One CTA partitions keys[0..n) in place, n * sizeof(T) a multiple of 16 and
// keys 16-byte aligned: one bulk asynchronous copy (TMA) stages the range in
// shared memory; predecessors are ranked by warp ballots in index order (a
// count pass, a scan of the per-(chunk, warp) counts, a scatter pass), which
// makes the partition stable; the stores of a warp fall in at most two runs.
// Returns the predecessor count, or ~0u if the copy's wait gave up (status
// set).  `bar` is a CTA-wide mbarrier (count 1) and `parity` its phase.
template <typename T>
struct CtaBulk {
  static constexpr uint32_t Head = 4096;  // per-(chunk, warp) counts
  static constexpr uint32_t Keys =
      (uint32_t)((level_smem_bytes<T, false>() - Head) / sizeof(T)) / Tr<T, false>::A *
      Tr<T, false>::A;
};

// First half of a CTA's on-chip partition: stages keys[0..n) (16-byte
// aligned, n <= CtaBulk<T>::Keys) in shared memory with one bulk copy and
// ranks the predecessors by warp ballots in index order.  Returns their
// count, or ~0u if the copy's wait gave up (status set).
template <typename T>
__device__ uint32_t cta_bulk_stage(const T* __restrict__ keys, uint32_t n, T pivot,
                                   unsigned char* smem, uint64_t* bar, uint32_t& parity,
                                   uint32_t* status) {
  constexpr uint32_t NT = Tr<T, false>::Threads, W = NT / 32;
  constexpr uint32_t FULL = 0xffffffffu;
  static_assert(((CtaBulk<T>::Keys + NT - 1) / NT) * W * 4 + 4 <= CtaBulk<T>::Head,
                "count space");
  uint32_t* cnt = reinterpret_cast<uint32_t*>(smem);
  T* sk = reinterpret_cast<T*>(smem + CtaBulk<T>::Head);
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t bytes = n * (uint32_t)sizeof(T);
  if (tid == 0) {
    fence_proxy_async_smem();  // this shared memory was last written by threads
    mbar_arrive_expect_tx(bar, bytes);
    for (uint32_t off = 0; off < bytes; off += 16384u) {
      const uint32_t len = bytes - off < 16384u ? bytes - off : 16384u;
      bulk_load(reinterpret_cast<unsigned char*>(sk) + off,
                reinterpret_cast<const unsigned char*>(keys) + off, len, bar);
    }
  }
  const bool ok = mbar_wait_bounded(bar, parity);
  if (!ok) {
    if (tid == 0) atomicOr(status, kStatTimeout | kSiteBulk);
    mbar_wait_bounded(bar, parity);  // let the copy land before the memory is reused
    __syncthreads();
    return ~0u;
  }
  parity ^= 1u;
  const uint32_t nch = (n + NT - 1) / NT;
  for (uint32_t c = 0; c < nch; c++) {
    const uint32_t q = c * NT + tid;
    const bool f = q < n && sk[q] <= pivot;
    const uint32_t bal = __ballot_sync(FULL, f);
    if (lane == 0) cnt[c * W + warp] = __popc(bal);
  }
  __syncthreads();
  if (warp == 0) {  // exclusive scan of the counts in (chunk, warp) order
    const uint32_t m = nch * W;
    uint32_t run = 0;
    for (uint32_t b0 = 0; b0 < m; b0 += 32) {
      const uint32_t v = b0 + lane < m ? cnt[b0 + lane] : 0u;
      uint32_t incl = v;
#pragma unroll
      for (uint32_t o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
      }
      if (b0 + lane < m) cnt[b0 + lane] = run + incl - v;
      run += __shfl_sync(FULL, incl, 31);
    }
    if (lane == 0) cnt[(CtaBulk<T>::Head / 4) - 1] = run;
  }
  __syncthreads();
  return cnt[(CtaBulk<T>::Head / 4) - 1];
}

// Second half: the staged keys' predecessors go to pred[0..) and their
// successors to succ[0..), each in index order (stable).  Ends with a CTA
// barrier (the shared memory may be reused at once).
template <typename T>
__device__ void cta_bulk_scatter(T* __restrict__ pred, T* __restrict__ succ, uint32_t n, T pivot,
                                 const unsigned char* smem) {
  constexpr uint32_t NT = Tr<T, false>::Threads, W = NT / 32;
  constexpr uint32_t FULL = 0xffffffffu;
  const uint32_t* cnt = reinterpret_cast<const uint32_t*>(smem);
  const T* sk = reinterpret_cast<const T*>(smem + CtaBulk<T>::Head);
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t nch = (n + NT - 1) / NT;
  for (uint32_t c = 0; c < nch; c++) {
    const uint32_t q = c * NT + tid;
    const T x = q < n ? sk[q] : pivot;
    const bool f = q < n && x <= pivot;
    const uint32_t bal = __ballot_sync(FULL, f);
    const uint32_t pre = cnt[c * W + warp] + __popc(bal & lt);  // predecessors before q
    if (q < n) {
      if (f) pred[pre] = x;
      else succ[q - pre] = x;
    }
  }
  __syncthreads();
}

// The whole on-chip partition of keys[0..n) by one CTA.  Returns the
// predecessor count, or ~0u if the copy's wait gave up (status set).  `bar`
// is a CTA-wide mbarrier (count 1) and `parity` its phase.
template <typename T>
__device__ uint32_t cta_partition_bulk(T* __restrict__ keys, uint32_t n, T pivot,
                                       unsigned char* smem, uint64_t* bar, uint32_t& parity,
                                       uint32_t* status) {
  const uint32_t total = cta_bulk_stage<T>(keys, n, pivot, smem, bar, parity, status);
  if (total == ~0u) return ~0u;
  cta_bulk_scatter<T>(keys, keys + total, n, pivot, smem);
  return total;
}

}  // namespace lp
