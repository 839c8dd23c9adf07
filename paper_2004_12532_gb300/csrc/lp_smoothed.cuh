// lp_smoothed.cuh -- the Smoothed Striding partial partition step on sm_103a
// (Sec. 4 of arXiv 2004.12532, "Formal Algorithm Description" and the figure
// "Smoothed Striding Algorithm").
//
// GPU mapping.  Each warp owns one group U_i at a time (the paper partitions
// every U_i serially, one processor per group).  The group's lines -- line
// j*g + (X[j]+i) mod g of every chunk j -- form a stream of nl lines in group
// order, which the warp partitions in place:
//   * lane 0 loads lines with 1-D bulk asynchronous copies (TMA) from both
//     ends of the stream, kQ lines in flight per side, each completing on an
//     mbarrier;
//   * every lane classifies one 16-byte vector of the consumed line; warp
//     ballots give each key its rank, and keys are appended to one of two
//     shared-memory rings (P: predecessors, S: successors);
//   * a full line of P is written back (bulk store) to the lowest line of the
//     stream not yet written, a full line of S to the highest, and only into
//     lines already consumed; the last one or two lines take what is left,
//     P first.
// Which end to consume next is decided by the slack of written-back lines on
// each side (lp_plan.h, StreamCtl), which keeps both rings bounded for any
// input.  Every line is read once and written once: one read and one write of
// every key, the I/O of the paper's Prop. 4.2.  The group ends predecessors
// first in its own slot order, exactly as the paper's serial partition leaves
// it, so k_i and v_i are the paper's.
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
  unsigned long long b, g;   // parameters used (g == 0: finished in one CTA)
  unsigned long long pad;
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
  static constexpr uint32_t LineBytes = kLineBytesMax;          // key bytes per line, max
  static constexpr uint32_t LineKeys = LineBytes / K;
  static constexpr uint32_t RingKeys = kRingLines * LineKeys;   // power of two
  static constexpr uint32_t V = 16u / K;                        // keys per 16-byte vector
  static constexpr uint32_t A = 16u / K;                        // alignment unit in keys
  static constexpr uint32_t Warps = KV ? 4u : 8u;               // groups in flight per CTA
  static constexpr uint32_t Threads = 32u * Warps;
  // one CTA partitions ranges up to this many keys in shared memory
  static constexpr uint32_t FinishKeys = kFinishBytes / (K + (KV ? 8u : 0u));
};

template <typename T, bool KV>
struct __align__(128) WarpSmem {
  T stage[kStages][Tr<T, KV>::LineKeys];
  T pring[Tr<T, KV>::RingKeys];
  T sring[Tr<T, KV>::RingKeys];
  uint64_t vstage[KV ? kStages : 1][KV ? Tr<T, KV>::LineKeys : 2];
  uint64_t vpring[KV ? Tr<T, KV>::RingKeys : 2];
  uint64_t vsring[KV ? Tr<T, KV>::RingKeys : 2];
  uint64_t bar[kStages];
  uint32_t tab_line[2 * kLineTab];   // issued lines: line index within the range
  uint32_t tab_len[2 * kLineTab];    // ... and its length in keys
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

// Partition group i of step G over the range starting at `base` (`vbase`
// for payloads).  Called by all 32 lanes of one warp with the same arguments;
// control is warp-uniform, lane 0 issues the bulk copies.  `phase` holds one
// parity bit per stage and persists across the warp's groups.  Returns false
// if a bounded wait gave up or a ring check failed (after draining the warp's
// copies in flight); k receives the group's predecessor count.
template <typename T, bool KV>
__device__ bool warp_stream_group(T* __restrict__ base, uint64_t* __restrict__ vbase,
                                  const StepGeom& G, uint64_t i, int64_t nl, T pivot,
                                  WarpSmem<T, KV>& sm, uint32_t& phase, uint64_t& k,
                                  uint32_t* status) {
  using R = Tr<T, KV>;
  constexpr uint32_t MASK = R::RingKeys - 1;
  constexpr uint32_t V = R::V;
  constexpr uint32_t FULL = 0xffffffffu;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t lt = (1u << lane) - 1u;
  k = 0;
  if (nl <= 0) return true;

  // X windows: lane l holds X[wf + l] (front) and X[wb - l] (back)
  int64_t wf = -64, wb = -64;
  uint64_t xf = 0, xb = 0;
  auto x_front = [&](int64_t m) -> uint64_t {
    if (G.strided) return 0;
    if (m < wf || m >= wf + 32) {
      wf = m;
      const uint64_t j = (uint64_t)wf + lane;
      xf = j < G.s ? range_of(sm_stream(G.sigma, j), G.g) : 0;
    }
    return __shfl_sync(FULL, xf, (int)(m - wf));
  };
  auto x_back = [&](int64_t m) -> uint64_t {
    if (G.strided) return 0;
    if (m > wb || m <= wb - 32) {
      wb = m;
      const int64_t j = wb - (int64_t)lane;
      xb = j >= 0 ? range_of(sm_stream(G.sigma, (uint64_t)j), G.g) : 0;
    }
    return __shfl_sync(FULL, xb, (int)(wb - m));
  };

  StreamCtl c;
  ctl_init(c, nl);

  auto issue = [&](int64_t line, uint32_t st, bool front) {
    const uint64_t x = front ? x_front(line) : x_back(line);
    uint64_t off = x + i;
    if (off >= G.g) off -= G.g;
    const uint64_t gl = (uint64_t)line * G.g + off;
    const uint32_t len = (uint32_t)line_len(G, gl);
    if (lane == 0) {
      const uint32_t slot = line_tab_slot_side(c, line, front);
      sm.tab_line[slot] = (uint32_t)gl;
      sm.tab_len[slot] = len;
      const uint32_t bytes = len * R::K;
      mbar_arrive_expect_tx(&sm.bar[st], KV ? 2u * bytes : bytes);
      bulk_load(&sm.stage[st][0], base + gl * G.b, bytes, &sm.bar[st]);
      if constexpr (KV) bulk_load(&sm.vstage[st][0], vbase + gl * G.b, bytes, &sm.bar[st]);
    }
  };
  auto flush = [&](const T* ring, const uint64_t* vring, uint64_t head, uint32_t gl,
                   uint32_t len) {
    // lane 0: ring[head .. head+len) -> line gl, split at the ring end
    const uint32_t off = (uint32_t)(head & MASK);
    const uint32_t first = min(len, R::RingKeys - off);
    T* dst = base + (uint64_t)gl * G.b;
    bulk_store(dst, ring + off, first * R::K);
    if constexpr (KV) bulk_store(vbase + (uint64_t)gl * G.b, vring + off, first * 8u);
    if (first < len) {
      bulk_store(dst + first, ring, (len - first) * R::K);
      if constexpr (KV) bulk_store(vbase + (uint64_t)gl * G.b + first, vring, (len - first) * 8u);
    }
    bulk_commit();
  };

  for (uint32_t q = 0; q < kQ; q++) {
    if (ctl_can_issue(c)) { issue(c.fi, stage_front(c.fi), true); c.fi++; }
    if (ctl_can_issue(c)) { issue(c.bi, stage_back(c, c.bi), false); c.bi--; }
  }
  __syncwarp();

  bool ok = true;
  while (!ctl_done(c)) {
    const bool front = ctl_pick_front(c);
    const int64_t line = front ? c.lo_c : c.hi_c;
    const bool from_front_q = line < c.fi;
    const uint32_t st = ctl_stage_of(c, line);
    const uint32_t len = sm.tab_len[line_tab_slot(c, line)];

    // ring capacity, counting bulk stores that may still read (uniform)
    if (ctl_p_count(c) + len + kPendingFlushes * G.b > R::RingKeys ||
        ctl_s_count(c) + len + kPendingFlushes * G.b > R::RingKeys) {
      if (lane == 0) atomicOr(status, kStatRing);
      ok = false;
      break;
    }
    const bool arrived = mbar_wait_bounded(&sm.bar[st], (phase >> st) & 1u);
    if (!__all_sync(FULL, arrived)) {
      if (lane == 0) atomicOr(status, kStatTimeout);
      ok = false;
      break;
    }
    phase ^= 1u << st;

    // classify: lane l takes vector l of the line
    const bool act = lane < len / V;
    T x[V];
    uint64_t y[V];
    uint32_t flags = 0;
    if (act) {
      load_vec<T>(&sm.stage[st][lane * V], x);
      if constexpr (KV) {
        const ulonglong2 w = *reinterpret_cast<const ulonglong2*>(&sm.vstage[st][lane * V]);
        y[0] = w.x; y[1] = w.y;
      }
#pragma unroll
      for (uint32_t v = 0; v < V; v++) flags |= (x[v] <= pivot ? 1u : 0u) << v;
    }
    uint32_t np = 0, pl = 0;
#pragma unroll
    for (uint32_t v = 0; v < V; v++) {
      const uint32_t bv = __ballot_sync(FULL, (flags >> v) & 1u);
      np += __popc(bv);
      pl += __popc(bv & lt);
    }
    if (act) {
      const uint32_t kl = lane * V;  // keys of the lanes below (all full vectors)
      uint64_t pp = c.p_tail + pl;
      uint64_t sp = c.s_tail + (kl - pl);
#pragma unroll
      for (uint32_t v = 0; v < V; v++) {
        if ((flags >> v) & 1u) {
          sm.pring[pp & MASK] = x[v];
          if constexpr (KV) sm.vpring[pp & MASK] = y[v];
          pp++;
        } else {
          sm.sring[sp & MASK] = x[v];
          if constexpr (KV) sm.vsring[sp & MASK] = y[v];
          sp++;
        }
      }
    }
    fence_proxy_async_smem();
    __syncwarp();  // ring writes visible to the copy engine; the stage is free

    c.p_tail += np;
    c.s_tail += len - np;
    c.k += np;
    if (front) c.lo_c++; else c.hi_c--;

    // refill the freed stage from the side it served
    if (ctl_can_issue(c)) {
      if (from_front_q) { issue(c.fi, stage_front(c.fi), true); c.fi++; }
      else { issue(c.bi, stage_back(c, c.bi), false); c.bi--; }
    }
    // write back full lines of P (front) and S (back) into consumed lines
    while (c.fw <= c.bw && ctl_consumed(c, c.fw)) {
      const uint32_t slot = line_tab_slot(c, c.fw);
      const uint32_t lw = sm.tab_len[slot];
      if (ctl_p_count(c) < lw) break;
      if (lane == 0) flush(sm.pring, sm.vpring, c.p_head, sm.tab_line[slot], lw);
      c.p_head += lw;
      c.fw++;
    }
    while (c.bw >= c.fw && ctl_consumed(c, c.bw)) {
      const uint32_t slot = line_tab_slot(c, c.bw);
      const uint32_t lw = sm.tab_len[slot];
      if (ctl_s_count(c) < lw) break;
      if (lane == 0) flush(sm.sring, sm.vsring, c.s_head, sm.tab_line[slot], lw);
      c.s_head += lw;
      c.bw--;
    }
    if (lane == 0) bulk_wait_read<kPendingFlushes>();
    __syncwarp();  // ring space of completed write-backs reusable
  }

  if (!ok) {
    // drain this warp's loads still in flight with bounded waits; the array
    // is left in an unspecified state and the status word says why
    if (lane == 0) {
      for (int64_t l = c.lo_c; l <= c.hi_c; l++) {
        if (l >= c.fi && l <= c.bi) continue;  // never issued
        const uint32_t s2 = ctl_stage_of(c, l);
        mbar_wait_bounded(&sm.bar[s2], (phase >> s2) & 1u);
      }
      bulk_wait_all<0>();
    }
    __syncwarp();
    return false;
  }

  // the last unwritten lines fw..bw take the rest of P, then the rest of S
  const uint64_t pc = ctl_p_count(c), sc = ctl_s_count(c), rem = pc + sc;
  for (uint64_t q = lane; q < rem; q += 32) {
    const bool isp = q < pc;
    const uint64_t r = isp ? ((c.p_head + q) & MASK) : ((c.s_head + (q - pc)) & MASK);
    const int64_t m = c.fw + (int64_t)(q / G.b);
    const uint64_t off = q % G.b;
    const uint64_t gw = sm.tab_line[line_tab_slot(c, m)];
    base[gw * G.b + off] = isp ? sm.pring[r] : sm.sring[r];
    if constexpr (KV) vbase[gw * G.b + off] = isp ? sm.vpring[r] : sm.vsring[r];
  }
  k = c.k;
  if (lane == 0) bulk_wait_read<0>();
  __syncwarp();  // rings and table free for the next group
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
  for (uint32_t q = tid; q < n; q += NT) {
    sk[q] = keys[q];
    if constexpr (KV) sv[q] = vals[q];
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

}  // namespace lp
