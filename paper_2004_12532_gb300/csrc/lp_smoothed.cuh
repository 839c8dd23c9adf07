// lp_smoothed.cuh -- the Smoothed Striding partial partition step on sm_103a
// (Sec. 4 of arXiv 2004.12532, "Formal Algorithm Description" and the figure
// "Smoothed Striding Algorithm").
//
// GPU mapping.  One CTA owns one group U_i at a time.  The group's lines
// (line j*g + (X[j]+i) mod g of every chunk j) are a stream of nl lines in
// group order; the CTA partitions that stream in place with two bulk-copy
// load queues (front and back, kQ lines in flight each), two shared-memory
// rings (P for predecessors, S for successors) and bulk-copy stores that write
// a full line of P to the lowest unwritten line and a full line of S to the
// highest, always into lines already read.  The serial partition of each U_i
// in the paper becomes this CTA-wide stream partition; it produces the same
// k_i and hence the same v_i.  Per-line ranks come from warp shuffles and a
// CTA scan of warp totals.  v_min / v_max are reduced with 64-bit atomic
// min / max into the level descriptor (order-independent, deterministic).
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
  unsigned long long b, g;   // parameters used
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
  int force_finish;          // one group (a plain CTA-wide partition)
};

template <typename T, bool KV>
struct Tr {
  static constexpr uint32_t K = sizeof(T);
  static constexpr uint32_t LineBytes = KV ? 2048u : 4096u;  // key bytes per line, max
  static constexpr uint32_t LineKeys = LineBytes / K;
  static constexpr uint32_t RingKeys = 8u * LineKeys;        // power of two
  static constexpr uint32_t V = 16u / K;                     // keys per 16-byte vector
  static constexpr uint32_t A = 16u / K;                     // alignment unit in keys
};

template <typename T, bool KV>
struct __align__(128) StreamSmem {
  T stage[kStages][Tr<T, KV>::LineKeys];
  T pring[Tr<T, KV>::RingKeys];
  T sring[Tr<T, KV>::RingKeys];
  uint64_t vstage[KV ? kStages : 1][KV ? Tr<T, KV>::LineKeys : 2];
  uint64_t vpring[KV ? Tr<T, KV>::RingKeys : 2];
  uint64_t vsring[KV ? Tr<T, KV>::RingKeys : 2];
  uint64_t bar[kStages];
  uint32_t warp_cnt[kThreads / 32];
  uint32_t abort_flag;
};

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

// Partition group i of the step G over the range starting at `base`
// (and `vbase` for payloads).  All threads of the CTA call this with the same
// arguments.  Returns the group's predecessor count in k (uniform).
// `phase` holds one parity bit per stage and persists across groups.
template <typename T, bool KV>
__device__ void stream_group(T* __restrict__ base, uint64_t* __restrict__ vbase,
                             const StepGeom& G, uint64_t i, int64_t nl, T pivot,
                             StreamSmem<T, KV>& sm, uint32_t& phase, uint64_t& k,
                             uint32_t* status) {
  using R = Tr<T, KV>;
  constexpr uint32_t MASK = R::RingKeys - 1;
  constexpr uint32_t V = R::V;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;

  StreamCtl c;
  ctl_init(c, nl);
  k = 0;
  if (nl <= 0) return;

  auto issue = [&](int64_t line, uint32_t st) {
    // thread 0 only
    uint64_t gl = group_line(G, i, (uint64_t)line);
    uint32_t len = (uint32_t)line_len(G, gl);
    uint32_t bytes = len * R::K;
    mbar_arrive_expect_tx(&sm.bar[st], KV ? 2u * bytes : bytes);
    bulk_load(&sm.stage[st][0], base + gl * G.b, bytes, &sm.bar[st]);
    if constexpr (KV) bulk_load(&sm.vstage[st][0], vbase + gl * G.b, bytes, &sm.bar[st]);
  };
  auto flush = [&](const T* ring, const uint64_t* vring, uint64_t head, uint64_t gl,
                   uint32_t len) {
    // thread 0 only: ring[head .. head+len) -> line gl, split at the ring end
    uint32_t off = (uint32_t)(head & MASK);
    uint32_t first = min(len, R::RingKeys - off);
    bulk_store(base + gl * G.b, ring + off, first * R::K);
    if constexpr (KV) bulk_store(vbase + gl * G.b, vring + off, first * 8u);
    if (first < len) {
      bulk_store(base + gl * G.b + first, ring, (len - first) * R::K);
      if constexpr (KV) bulk_store(vbase + gl * G.b + first, vring, (len - first) * 8u);
    }
    bulk_commit();
  };

  // initial loads: kQ from each end, alternating
  for (uint32_t q = 0; q < kQ; q++) {
    if (ctl_can_issue(c)) {
      if (tid == 0) issue(c.fi, stage_front(c.fi));
      c.fi++;
    }
    if (ctl_can_issue(c)) {
      if (tid == 0) issue(c.bi, stage_back(c, c.bi));
      c.bi--;
    }
  }

  bool aborted = false;
  while (!ctl_done(c)) {
    const bool front = ctl_pick_front(c);
    const int64_t line = front ? c.lo_c : c.hi_c;
    const bool from_front_q = line < c.fi;
    const uint32_t st = ctl_stage_of(c, line);
    const uint64_t gl = group_line(G, i, (uint64_t)line);
    const uint32_t len = (uint32_t)line_len(G, gl);

    // ring capacity (pending flushes included); uniform check
    if (ctl_p_count(c) + len + kPendingFlushes * G.b > R::RingKeys ||
        ctl_s_count(c) + len + kPendingFlushes * G.b > R::RingKeys) {
      if (tid == 0) {
        atomicOr(status, kStatRing);
        sm.abort_flag = 1u;
      }
      aborted = true;
      break;
    }

    if (!mbar_wait_bounded(&sm.bar[st], (phase >> st) & 1u)) sm.abort_flag = 1u;

    // classify one 16-byte vector per thread
    const uint32_t nvec = len / V;
    const bool act = tid < nvec;
    T x[V];
    uint64_t y[V];
    uint32_t flags = 0, cnt = 0;
    if (act) {
      load_vec<T>(&sm.stage[st][tid * V], x);
      if constexpr (KV) {
        ulonglong2 w = *reinterpret_cast<const ulonglong2*>(&sm.vstage[st][tid * V]);
        y[0] = w.x; y[1] = w.y;
      }
#pragma unroll
      for (uint32_t v = 0; v < V; v++) {
        uint32_t f = x[v] <= pivot ? 1u : 0u;
        flags |= f << v;
        cnt += f;
      }
    }
    uint32_t incl = cnt;
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) sm.warp_cnt[warp] = incl;
    __syncthreads();  // (1) warp totals and abort flag visible
    if (sm.abort_flag) {
      if (tid == 0) atomicOr(status, kStatTimeout);
      aborted = true;
      break;
    }
    phase ^= 1u << st;  // this stage's load has been consumed
    uint32_t wbase = 0, total = 0;
#pragma unroll
    for (uint32_t w = 0; w < kThreads / 32; w++) {
      uint32_t cw = sm.warp_cnt[w];
      wbase += (w < warp) ? cw : 0u;
      total += cw;
    }
    if (act) {
      const uint32_t excl = wbase + incl - cnt;
      uint64_t pp = c.p_tail + excl;
      uint64_t sp = c.s_tail + (uint64_t)tid * V - excl;
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
    __syncthreads();  // (2) ring writes visible to the bulk-copy engine; stage free

    c.p_tail += total;
    c.s_tail += len - total;
    c.k += total;
    if (front) c.lo_c++; else c.hi_c--;

    // refill the freed stage from the side it served
    if (ctl_can_issue(c)) {
      if (from_front_q) {
        if (tid == 0) issue(c.fi, stage_front(c.fi));
        c.fi++;
      } else {
        if (tid == 0) issue(c.bi, stage_back(c, c.bi));
        c.bi--;
      }
    }
    // write back full lines of P (front) and S (back) into consumed lines
    while (c.fw <= c.bw && ctl_consumed(c, c.fw)) {
      const uint64_t gw = group_line(G, i, (uint64_t)c.fw);
      const uint32_t lw = (uint32_t)line_len(G, gw);
      if (ctl_p_count(c) < lw) break;
      if (tid == 0) flush(sm.pring, sm.vpring, c.p_head, gw, lw);
      c.p_head += lw;
      c.fw++;
    }
    while (c.bw >= c.fw && ctl_consumed(c, c.bw)) {
      const uint64_t gw = group_line(G, i, (uint64_t)c.bw);
      const uint32_t lw = (uint32_t)line_len(G, gw);
      if (ctl_s_count(c) < lw) break;
      if (tid == 0) flush(sm.sring, sm.vsring, c.s_head, gw, lw);
      c.s_head += lw;
      c.bw--;
    }
    if (tid == 0) bulk_wait_read<kPendingFlushes>();
  }

  if (aborted) {
    // drain this CTA's own loads still in flight, with bounded waits; the
    // array is left in an unspecified state and the status word says why
    if (tid == 0) {
      for (int64_t l = c.lo_c; l <= c.hi_c; l++) {
        if (l >= c.fi && l <= c.bi) continue;  // never issued
        uint32_t st = ctl_stage_of(c, l);
        mbar_wait_bounded(&sm.bar[st], (phase >> st) & 1u);
      }
      bulk_wait_all<0>();
    }
    __syncthreads();
    k = c.k;
    return;
  }

  // the last unwritten lines fw..bw take the rest of P, then the rest of S
  const uint64_t pc = ctl_p_count(c), sc = ctl_s_count(c), rem = pc + sc;
  for (uint64_t q = tid; q < rem; q += kThreads) {
    const bool isp = q < pc;
    const uint64_t r = isp ? ((c.p_head + q) & MASK) : ((c.s_head + (q - pc)) & MASK);
    const uint64_t m = (uint64_t)c.fw + q / G.b;
    const uint64_t off = q % G.b;
    const uint64_t gw = group_line(G, i, m);
    base[gw * G.b + off] = isp ? sm.pring[r] : sm.sring[r];
    if constexpr (KV) vbase[gw * G.b + off] = isp ? sm.vpring[r] : sm.vsring[r];
  }
  if (tid == 0) bulk_wait_read<0>();
  __syncthreads();  // rings free for the next group
  k = c.k;
}

}  // namespace lp
