// lp_batched.cu -- many independent partitions in one persistent cooperative
// launch.  Each segment is partitioned by the Recursive Smoothed Striding
// scheme of Sec. 4: Partial Partition Steps on its open range [v_min, v_max)
// until the range is empty.
//
// The kernel works in rounds, with grid barriers between phases:
//   plan  every CTA takes a slice of the segments: the last step's v_min /
//         v_max become the open range; an empty range finishes the segment
//         (its unaligned head and tail are put in place, the split written);
//         a residual range (after the first step) that one CTA's shared
//         memory holds becomes a CTA task (the base case, finished on chip);
//         one that more than one CTA (up to the grid) holds becomes a
//         multi-CTA finish: that many CTAs stage a slice each, count, and
//         once all of the range is on chip write a stable partition of it;
//         a first range of at most warp_cap keys gets a one-group step (g = 1:
//         one warp partitions the whole range, as the paper's base case
//         partitions serially); a larger one a step with g groups from the
//         parameter rule.  Grid barrier; every CTA places its slice's tasks:
//         CTA tasks and one-group segments in lists, multi-group segments
//         with the prefix of their group counts.  Grid barrier.
//   tasks the multi-CTA finishes run first, their slices taken in order from
//         a counter; every CTA takes CTA tasks from another; then every warp takes
//         warp tasks from another -- the groups of multi-group segments first
//         (binary search over their prefix), then the one-group segments --
//         and partitions that group (warp_pair_group, as in the single
//         partition); v_i go to the segment's record by atomic min / max.
//         Grid barrier.  A round whose tasks were all on-chip finishes is
//         the last: each CTA then places the heads and tails of its slice's
//         segments itself.
// A segment's steps depend on its own size and state only (never on what it
// is batched with), so its result is the same in any batch.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lp_batch_init.cuh"
#include "lp_batched.h"
#include "lp_coop.cuh"
#include "lp_fixup.cuh"
#include "lp_launch.h"

namespace lp {

namespace {

// Segment fields written by other CTAs are read through L2, never from L1.
__device__ __forceinline__ uint64_t L2(const uint64_t& x) {
  return __ldcg(reinterpret_cast<const unsigned long long*>(&x));
}
__device__ __forceinline__ unsigned long long L2(const unsigned long long& x) { return __ldcg(&x); }
__device__ __forceinline__ uint32_t L2(const uint32_t& x) {
  return __ldcg(reinterpret_cast<const unsigned int*>(&x));
}

template <typename T>
__global__ void __launch_bounds__(Tr<T, false>::Threads) batched_kernel(SegDesc* segs,
                                                                        uint32_t count,
                                                                        BatchArgs a,
                                                                        BatchScratch B) {
  using R = Tr<T, false>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ unsigned int flag;
  constexpr int KP = (int)kPlanKinds;
  __shared__ uint32_t wsum[KP][R::Warps];
  __shared__ uint32_t base_s[KP];
  __shared__ unsigned long long tot_s[KP];
  __shared__ uint32_t fetch;
  __shared__ __align__(8) uint64_t cta_bar;  // the CTA tasks' bulk copies
  uint32_t cta_parity = 0;
  const uint32_t cta_cap = CtaBulk<T>::Keys;
  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;
  WarpSmem<T, false>& ws = reinterpret_cast<WarpSmem<T, false>*>(smem_raw)[warp];
  uint32_t phase = 0;
  TaskScratch S;
  S.status = B.status;
  S.bar = B.bar;
  // this CTA's slice of the segments
  const uint32_t s_lo = (uint32_t)((uint64_t)count * blockIdx.x / gridDim.x);
  const uint32_t s_hi = (uint32_t)((uint64_t)count * (blockIdx.x + 1) / gridDim.x);
  if (lane == 0) {
    for (uint32_t st = 0; st < R::Stages; st++) mbar_init(&ws.bar[st], 1);
    if (tid == 0) mbar_init(&cta_bar, 1);
    fence_mbar_init();
    fence_proxy_async_smem();
  }
  __syncthreads();

  // CTA-wide exclusive scan of (single, groups, multi, cta, multi-CTA slices,
  // multi-CTA segments) over the slice in chunks of R::Threads; this thread's
  // offsets and the chunk totals
  auto cta_scan = [&](const uint32_t (&in)[KP], uint32_t (&ex)[KP], uint32_t (&tot)[KP]) {
#pragma unroll
    for (int c = 0; c < KP; c++) {
      uint32_t v = in[c];
#pragma unroll
      for (uint32_t o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
      }
      if (lane == 31) wsum[c][warp] = v;
      ex[c] = v - in[c];
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < KP; c++) {
      uint32_t before = 0, all = 0;
      for (uint32_t w = 0; w < R::Warps; w++) {
        const uint32_t y = wsum[c][w];
        if (w < warp) before += y;
        all += y;
      }
      ex[c] += before;
      tot[c] = all;
    }
    __syncthreads();
  };

  // grid barrier; false (status set) if this CTA gave up waiting
  auto sync_grid = [&]() -> bool {
    if (grid_barrier(S.bar, gridDim.x, &flag)) return true;
    if (tid == 0) atomicOr(S.status, kStatTimeout | kSiteRounds);
    return false;
  };
  const bool stamp = blockIdx.x == 0 && tid == 0;
  for (uint32_t round = 0; round <= a.max_rounds; round++) {
    unsigned long long* tr = round < kBatchRoundSlots ? B.tround + 4 * round : nullptr;
    if (stamp && tr) tr[0] = global_timer_ns();
    // ------------------------------------------------------------ plan A
    // singles, multi groups, multi segments, CTA tasks, multi-CTA slices and segments
    uint32_t my[KP] = {0, 0, 0, 0, 0, 0};
    for (uint32_t c0 = s_lo; c0 < s_hi; c0 += R::Threads) {
      const uint32_t s = c0 + tid;
      uint32_t in[KP] = {0, 0, 0, 0, 0, 0};
      if (s < s_hi) {
        SegDesc& d = segs[s];
        if (L2(d.state) == kSegOpen) {
          const uint32_t level = L2(d.level);  // steps issued so far
          const uint64_t h = L2(d.h), be = L2(d.be), n = L2(d.n);
          uint64_t lo = L2(d.lo), hi = L2(d.hi);
          if (level > 0) {  // the last step left [vmin, vmax)
            lo = L2(d.vmin);
            hi = L2(d.vmax);
            if (level == 1) d.body_count = L2(d.count);
            if (lo < hi) {  // to the 16-byte grid of the body
              lo = h + ((lo - h) / R::A) * R::A;
              const uint64_t h2 = h + ((hi - h + R::A - 1) / R::A) * R::A;
              hi = h2 < be ? h2 : be;
            } else {
              lo = hi = 0;
            }
          }
          const uint64_t m = hi > lo ? hi - lo : 0;
          if (m == 0) {  // finished: head and tail, then the split
            const unsigned long long t = seg_fixup<T>(
                reinterpret_cast<T*>(d.keys), n, h, be,
                level > 0 ? (unsigned long long)L2(d.body_count) : 0ull, (T)L2(d.pivot));
            d.t = t;
            a.splits[s] = t;
            d.state = kSegDone;
          } else {
            d.lo = lo;
            d.hi = hi;
            if (level > 0 && m <= cta_cap) {
              // a residual range one CTA holds: finished on chip (a CTA task);
              // first ranges that small stay one-warp steps, which many
              // small segments keep busy in parallel
              atomicAdd(&B.totals[2], (unsigned long long)m);  // keys this round streams
              d.g = 0;
              d.b = 1;
              in[3] = 1;
            } else if (level > 0 && m <= (uint64_t)a.mc_slices * cta_cap) {
              // a residual range c > 1 CTAs hold: finished on chip by c
              // CTAs, a stable partition (the same as one CTA's); its keys
              // are counted when it runs
              const uint64_t c = (m + cta_cap - 1) / cta_cap;
              d.g = 0;
              d.b = c;
              d.t = 0ull;  // slices done
              d.staged = 0u;
              in[4] = (uint32_t)c;
              in[5] = 1;
            } else {
              atomicAdd(&B.totals[2], (unsigned long long)m);  // keys this round streams
              StepParams P = choose_params(m, R::K, a.group_workers, a.line_bytes,
                                           level ? a.min_chunks_residual : a.min_chunks);
              if (m <= a.warp_cap || level + 1 >= a.max_rounds) P.g = 1;
              d.b = P.b;
              d.g = P.g;
              d.vmin = ~0ull;
              d.vmax = 0ull;
              d.count = 0ull;
              d.level = level + 1;
              if (P.g == 1) in[0] = 1;
              else { in[1] = (uint32_t)P.g; in[2] = 1; }
            }
          }
        }
      }
      uint32_t ex[KP], tot[KP];
      cta_scan(in, ex, tot);
#pragma unroll
      for (int c = 0; c < KP; c++) my[c] += tot[c];
    }
    if (tid < KP) B.cta_tot[KP * blockIdx.x + tid] = my[tid];
    if (!sync_grid()) return;

    // ------------------------------------------------------------ plan B
    // this CTA's offsets: the totals of the CTAs before it; and the grand totals
    {
      uint32_t before[KP] = {0, 0, 0, 0, 0, 0}, all[KP] = {0, 0, 0, 0, 0, 0};
      for (uint32_t c = tid; c < gridDim.x; c += R::Threads) {
#pragma unroll
        for (int q = 0; q < KP; q++) {
          const uint32_t y = __ldcg(&B.cta_tot[KP * c + q]);
          if (c < blockIdx.x) before[q] += y;
          all[q] += y;
        }
      }
#pragma unroll
      for (int q = 0; q < KP; q++) {
#pragma unroll
        for (uint32_t o = 16; o > 0; o >>= 1) {
          before[q] += __shfl_xor_sync(0xffffffffu, before[q], o);
          all[q] += __shfl_xor_sync(0xffffffffu, all[q], o);
        }
        if (lane == 0) wsum[q][warp] = before[q];
      }
      __syncthreads();
      if (tid < KP) {
        uint32_t b = 0;
        for (uint32_t w = 0; w < R::Warps; w++) b += wsum[tid][w];
        base_s[tid] = b;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < KP; q++)
        if (lane == 0) wsum[q][warp] = all[q];
      __syncthreads();
      if (tid < KP) {
        unsigned long long t = 0;
        for (uint32_t w = 0; w < R::Warps; w++) t += wsum[tid][w];
        tot_s[tid] = t;
      }
      __syncthreads();
    }
    uint32_t run[KP];
#pragma unroll
    for (int c = 0; c < KP; c++) run[c] = base_s[c];
    for (uint32_t c0 = s_lo; c0 < s_hi; c0 += R::Threads) {
      const uint32_t s = c0 + tid;
      uint32_t in[KP] = {0, 0, 0, 0, 0, 0};
      if (s < s_hi && L2(segs[s].state) == kSegOpen) {
        const uint64_t g = L2(segs[s].g);
        if (g == 0) {
          const uint64_t c = L2(segs[s].b);
          if (c <= 1) in[3] = 1;
          else { in[4] = (uint32_t)c; in[5] = 1; }
        } else if (g == 1) {
          in[0] = 1;
        } else {
          in[1] = (uint32_t)g;
          in[2] = 1;
        }
      }
      uint32_t ex[KP], tot[KP];
      cta_scan(in, ex, tot);
      if (in[0]) B.singles[run[0] + ex[0]] = s;
      if (in[2]) {
        B.mprefix[run[2] + ex[2]] = run[1] + ex[1];
        B.mseg[run[2] + ex[2]] = s;
      }
      if (in[3]) B.ctalist[run[3] + ex[3]] = s;
      if (in[5]) {
        B.mcprefix[run[5] + ex[5]] = run[4] + ex[4];
        B.mcseg[run[5] + ex[5]] = s;
      }
#pragma unroll
      for (int c = 0; c < KP; c++) run[c] += tot[c];
    }
    const unsigned long long n_single = tot_s[0], w_multi = tot_s[1];
    const uint32_t n_multi = (uint32_t)tot_s[2], n_cta = (uint32_t)tot_s[3];
    const uint32_t n_mcslots = (uint32_t)tot_s[4], n_mc = (uint32_t)tot_s[5];
    if (blockIdx.x == 0 && tid == 0) {
      B.mprefix[n_multi] = w_multi;
      B.mcprefix[n_mc] = n_mcslots;
      B.counters[0] = 0u;
      B.counters[1] = 0u;
      B.counters[2] = 0u;
      B.counters[3] = 0u;
      __threadfence();
    }
    if (!sync_grid()) return;
    if (n_single == 0 && w_multi == 0 && n_cta == 0 && n_mc == 0) break;  // all done

    // ------------------------------------------------------------ tasks
    const unsigned long long W = w_multi + n_single;
    if (stamp && tr) {
      tr[1] = global_timer_ns();
      tr[3] = W + n_cta + n_mcslots;
    }
    if (n_cta > 0 || n_mc > 0) {  // CTA tasks first: they use the warps' shared memory
      if (lane == 0)
        for (uint32_t st = 0; st < R::Stages; st++) mbar_inval(&ws.bar[st]);
      __syncthreads();
      // multi-CTA finishes.  CTAs take slices in slice order from a counter;
      // each stages and counts its slice, adds it to its finish's staged
      // count and waits until every slice of the finish is staged (all of the
      // range's keys on chip); then it writes its predecessors and successors
      // to their final places, and the last slice of a finish to complete
      // places the head and tail.  A finish has at most a.mc_slices <=
      // gridDim.x slices and a CTA holds one slice at a time, taken in order
      // (all CTAs resident: a cooperative launch), so the slices a CTA
      // waits for are taken by CTAs that wait for nothing else: every wait
      // ends.  The counts live in windows of a.mc_window slices (at least
      // any finish's), grid barriers between; a finish cut by a window's end
      // starts the next.
      // the last finish starting at or before slot: a 32-way search, one
      // probe per lane (the starts increase), a few dependent loads deep
      auto finish_of = [&](uint32_t slot) {
        uint32_t lo_k = 0, hi_k = n_mc;
        while (hi_k - lo_k > 1) {
          const uint32_t step = (hi_k - lo_k + 31) / 32;
          const uint32_t q = lo_k + (lane + 1) * step;
          const bool le = q < hi_k && __ldcg(&B.mcprefix[q]) <= slot;
          const uint32_t below = __popc(__ballot_sync(0xffffffffu, le));
          lo_k += below * step;
          const uint32_t h = lo_k + step;
          hi_k = h < hi_k ? h : hi_k;
        }
        return lo_k;
      };
      uint32_t win = 0;
      for (uint32_t w0 = 0; w0 < n_mcslots; win++) {
        uint32_t wend = n_mcslots - w0 > a.mc_window ? w0 + a.mc_window : n_mcslots;
        if (wend < n_mcslots) {
          const uint32_t kc = finish_of(wend - 1);
          const uint32_t pc = __ldcg(&B.mcprefix[kc]);
          if (__ldcg(&B.mcprefix[kc + 1]) > wend) wend = pc;
        }
        if (wend <= w0) {  // a finish longer than a window: never planned, never run
          if (tid == 0) atomicOr(S.status, kStatTimeout | kSiteRounds);
          return;
        }
        uint32_t* const claim = &B.counters[2 + (win & 1u)];
        // the next window's counter: every CTA took its last slice from it
        // before the barrier that opened this window
        if (blockIdx.x == 0 && tid == 0) B.counters[2 + ((win + 1u) & 1u)] = 0u;
        for (;;) {
          if (tid == 0) fetch = atomicAdd(claim, 1u);
          __syncthreads();
          const uint32_t slot = w0 + fetch;
          __syncthreads();
          if (slot >= wend) break;
          const uint32_t k = finish_of(slot);
          const uint32_t p = __ldcg(&B.mcprefix[k]);
          const uint32_t c = __ldcg(&B.mcprefix[k + 1]) - p;
          const uint32_t s = __ldcg(&B.mcseg[k]);
          SegDesc& d = segs[s];
          T* keys = reinterpret_cast<T*>(d.keys);
          const T pivot = (T)L2(d.pivot);
          const uint64_t lo = L2(d.lo), m = L2(d.hi) - lo;
          const uint64_t w = ((m + c - 1) / c + R::A - 1) / R::A * R::A;
          const uint64_t a0 = min(m, (uint64_t)(slot - p) * w);
          const uint64_t nj = min(m, a0 + w) - a0;
          uint32_t got = 0;
          if (nj > 0)
            got = cta_bulk_stage<T>(keys + lo + a0, (uint32_t)nj, pivot, smem_raw, &cta_bar,
                                    cta_parity, S.status);
          // publish the count, then wait for the finish's other slices
          fence_proxy_async_global();
          __syncthreads();
          if (tid == 0) {
            B.mccount[slot - w0] = got == ~0u ? 0u : got;
            __threadfence();
            atomicAdd(&d.staged, 1u);
            bool ok = got != ~0u;
            const volatile uint32_t* sv = &d.staged;
            const uint64_t t0 = global_timer_ns();
            while (*sv < c) {
              if (global_timer_ns() - t0 > kWaitLimitNs) {
                atomicOr(S.status, kStatTimeout | kSiteRounds);
                ok = false;
                break;
              }
              __nanosleep(32);
            }
            __threadfence();
            // a slice that could not be staged leaves the finish unwritten
            if (ok && (*reinterpret_cast<volatile uint32_t*>(S.status) & kStatTimeout)) ok = false;
            flag = ok ? 1u : 0u;
          }
          __syncthreads();
          fence_proxy_async_global();
          if (!flag) break;
          // predecessors of the slices before this one, and of the whole range
          unsigned long long before = 0, all = 0;
          for (uint32_t q = tid; q < c; q += R::Threads) {
            const uint32_t y = __ldcg(&B.mccount[p - w0 + q]);
            all += y;
            if (p + q < slot) before += y;
          }
#pragma unroll
          for (uint32_t o = 16; o > 0; o >>= 1) {
            before += __shfl_xor_sync(0xffffffffu, before, o);
            all += __shfl_xor_sync(0xffffffffu, all, o);
          }
          if (lane == 0) {
            wsum[0][warp] = (uint32_t)before;
            wsum[1][warp] = (uint32_t)all;
          }
          __syncthreads();
          uint64_t pb = 0, pt = 0;
          for (uint32_t w2 = 0; w2 < R::Warps; w2++) {
            pb += wsum[0][w2];
            pt += wsum[1][w2];
          }
          if (nj > 0)
            cta_bulk_scatter<T>(keys + lo + pb, keys + lo + pt + (a0 - pb), (uint32_t)nj, pivot,
                                smem_raw);
          __threadfence();
          __syncthreads();
          if (tid == 0) {
            if (slot == p) atomicAdd(&B.totals[2], (unsigned long long)m);  // keys streamed
            if (atomicAdd(&d.t, 1ull) + 1 == c) {  // the last slice: the others' writes are visible
              if (round < a.max_rounds) {  // the next plan places the head and tail
                d.vmin = lo;
                d.vmax = lo;
              } else {
                __threadfence();
                const unsigned long long t =
                    seg_fixup<T>(keys, L2(d.n), L2(d.h), L2(d.be), L2(d.body_count), pivot);
                d.t = t;
                a.splits[s] = t;
                d.state = kSegDone;
              }
            }
          }
          __syncthreads();
        }
        w0 = wend;
        if (w0 < n_mcslots && !sync_grid()) return;
      }
      // a residual range finished on chip leaves an empty open range: the
      // next round's plan (one thread per segment) puts its head and tail in
      // place and writes the split, off this CTA's path -- but not after the
      // last round
      const bool defer = round < a.max_rounds;
      uint32_t next = 0;
      if (tid == 0) next = atomicAdd(&B.counters[1], 1u);
      for (;;) {
        if (tid == 0) fetch = next;
        __syncthreads();
        const uint32_t c = fetch;
        __syncthreads();
        if (c >= n_cta) break;
        // the following task, taken now: the counter's latency hides behind this one
        if (tid == 0) next = atomicAdd(&B.counters[1], 1u);
        const uint32_t s = __ldcg(&B.ctalist[c]);
        SegDesc& d = segs[s];
        T* keys = reinterpret_cast<T*>(d.keys);
        const T pivot = (T)L2(d.pivot);
        const uint64_t lo = L2(d.lo), hi = L2(d.hi);
        const uint32_t cnt = cta_partition_bulk<T>(keys + lo, (uint32_t)(hi - lo), pivot,
                                                   smem_raw, &cta_bar, cta_parity, S.status);
        if (cnt == ~0u) break;  // a wait gave up (status set)
        if (tid == 0) {
          if (defer && L2(d.level) > 0) {
            d.vmin = lo;
            d.vmax = lo;
          } else {
            __threadfence_block();
            // a first-level CTA task partitioned the whole body
            const unsigned long long bc = L2(d.level) == 0 ? cnt : L2(d.body_count);
            const unsigned long long t =
                seg_fixup<T>(keys, L2(d.n), L2(d.h), L2(d.be), bc, pivot);
            d.t = t;
            a.splits[s] = t;
            d.state = kSegDone;
          }
        }
        __syncthreads();
      }
      if (lane == 0) {
        for (uint32_t st = 0; st < R::Stages; st++) mbar_init(&ws.bar[st], 1);
        fence_mbar_init();
        fence_proxy_async_smem();
      }
      __syncwarp();
      phase = 0;
    }
    for (;;) {
      uint32_t k = 0;
      if (lane == 0) k = atomicAdd(&B.counters[0], 1u);
      k = __shfl_sync(0xffffffffu, k, 0);
      if (k >= W) break;
      uint32_t s, i;
      if (k < w_multi) {  // a group of a multi-group segment: the last entry <= k
        uint32_t lo_s = 0, hi_s = n_multi;
        while (hi_s - lo_s > 1) {
          const uint32_t mid = (lo_s + hi_s) >> 1;
          if (__ldcg(&B.mprefix[mid]) <= k) lo_s = mid; else hi_s = mid;
        }
        s = __ldcg(&B.mseg[lo_s]);
        i = (uint32_t)(k - __ldcg(&B.mprefix[lo_s]));
      } else {
        s = __ldcg(&B.singles[k - w_multi]);
        i = 0;
      }
      SegDesc& d = segs[s];
      const uint64_t lo = L2(d.lo), hi = L2(d.hi);
      const uint64_t b = L2(d.b), g = L2(d.g);
      const uint32_t lev = L2(d.level);
      const StepGeom G = make_geom(hi - lo, b, g, level_seed(L2(d.seed), lev), 0);
      T* base = reinterpret_cast<T*>(d.keys) + lo;
      const int32_t nl = (int32_t)group_num_lines(G, i);
      uint64_t kk = 0;
      if (!warp_pair_group<T, false>(base, nullptr, G, i, nl, (T)L2(d.pivot), ws, phase, kk,
                                     S.status))
        break;
      if (nl > 0 && lane == 0) {
        const unsigned long long v = lo + group_split_pos(G, i, (uint64_t)nl, kk);
        atomicMin(&d.vmin, v);
        atomicMax(&d.vmax, v);
        atomicAdd(&d.count, (unsigned long long)kk);
      }
    }
    __syncwarp();
    if (!sync_grid()) return;
    if (stamp && tr) tr[2] = global_timer_ns();
    if (n_single == 0 && w_multi == 0) {
      // only on-chip finishes ran: every segment still open has an empty open
      // range, so what a further plan would do is this -- its head and tail
      // put in place, its split written -- with no grid barrier after it
      for (uint32_t s = s_lo + tid; s < s_hi; s += R::Threads) {
        SegDesc& d = segs[s];
        if (L2(d.state) != kSegOpen) continue;
        const unsigned long long t =
            seg_fixup<T>(reinterpret_cast<T*>(d.keys), L2(d.n), L2(d.h), L2(d.be),
                         L2(d.body_count), (T)L2(d.pivot));
        d.t = t;
        a.splits[s] = t;
        d.state = kSegDone;
      }
      break;
    }
  }
  __syncthreads();
  if (lane == 0) {
    for (uint32_t st = 0; st < R::Stages; st++) mbar_inval(&ws.bar[st]);
    if (tid == 0) mbar_inval(&cta_bar);
  }
}

// Per-segment set-up on the device: the 16-byte aligned body of each segment.
template <typename T>
__global__ void batch_setup_kernel(SegDesc* segs, uint32_t count, uint64_t seed,
                                   unsigned long long* traffic, unsigned long long* tround,
                                   uint32_t* bar) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  batch_launch_reset(traffic, tround, bar, s);
  if (s >= count) return;
  batch_seg_init<T>(segs[s], seed);
}

}  // namespace

namespace {
size_t up256(size_t b) { return (b + 255) / 256 * 256; }
}  // namespace

size_t batch_scratch_bytes(uint32_t count) {
  return up256(((size_t)count + 1) * 8) + 3 * up256((size_t)count * 4) +
         up256(((size_t)count + 1) * 4) + up256((size_t)count * 4) +
         up256((size_t)kMcWindow * 4) + up256((size_t)kBatchMaxGrid * kPlanKinds * 4) +
         up256(kBatchRoundSlots * 4 * 8) + 256;
}

BatchScratch carve_batch_scratch(void* base, uint32_t count, uint32_t* bar, uint32_t* status) {
  unsigned char* p = static_cast<unsigned char*>(base);
  BatchScratch B;
  B.mprefix = reinterpret_cast<unsigned long long*>(p);
  p += up256(((size_t)count + 1) * 8);
  B.mseg = reinterpret_cast<uint32_t*>(p);
  p += up256((size_t)count * 4);
  B.singles = reinterpret_cast<uint32_t*>(p);
  p += up256((size_t)count * 4);
  B.ctalist = reinterpret_cast<uint32_t*>(p);
  p += up256((size_t)count * 4);
  B.mcprefix = reinterpret_cast<uint32_t*>(p);
  p += up256(((size_t)count + 1) * 4);
  B.mcseg = reinterpret_cast<uint32_t*>(p);
  p += up256((size_t)count * 4);
  B.mccount = reinterpret_cast<uint32_t*>(p);
  p += up256((size_t)kMcWindow * 4);
  B.cta_tot = reinterpret_cast<uint32_t*>(p);
  p += up256((size_t)kBatchMaxGrid * kPlanKinds * 4);
  B.tround = reinterpret_cast<unsigned long long*>(p);
  p += up256(kBatchRoundSlots * 4 * 8);
  B.totals = reinterpret_cast<unsigned long long*>(p);
  B.counters = reinterpret_cast<uint32_t*>(p + 64);
  B.bar = bar;
  B.status = status;
  return B;
}

template <typename T>
cudaError_t launch_batched(SegDesc* d_segs, uint32_t count, uint64_t seed, uint64_t* d_splits,
                           const BatchScratch& Bs, const BatchTuning& tune, LaunchCfg& cfg,
                           bool records_ready) {
  using R = Tr<T, false>;
  cudaStream_t st = cfg.stream;
  if (count == 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  if (!records_ready) {
    const uint32_t setup_threads = count > kBatchRoundSlots * 4 ? count : kBatchRoundSlots * 4;
    batch_setup_kernel<T><<<(setup_threads + 255) / 256, 256, 0, st>>>(d_segs, count, seed,
                                                                        Bs.totals + 2, Bs.tround,
                                                                        Bs.bar);
    cfg.launches++;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  BatchArgs a;
  a.splits = d_splits;
  a.max_rounds = kMaxLevels;
  uint32_t grid = cfg.grid;
  if (tune.ctas && tune.ctas < grid) grid = tune.ctas;
  if (grid > kBatchMaxGrid) grid = kBatchMaxGrid;
  a.group_workers = tune.group_workers ? tune.group_workers : (uint64_t)grid * R::Warps;
  a.line_bytes = tune.line_bytes && tune.line_bytes < R::LineBytes ? tune.line_bytes
                                                                  : R::LineBytes;
  a.min_chunks = tune.min_chunks ? tune.min_chunks : 32;
  a.warp_cap = kWarpCapBytes / R::K;
  a.min_chunks_residual = tune.min_chunks_residual ? tune.min_chunks_residual : a.min_chunks;
  a.mc_slices = tune.mc_slices && tune.mc_slices < grid ? tune.mc_slices : grid;
  a.mc_window = a.mc_slices < grid ? 4 * a.mc_slices : kMcWindow;
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
                                              LaunchCfg&, bool);
template cudaError_t launch_batched<uint32_t>(SegDesc*, uint32_t, uint64_t, uint64_t*,
                                              const BatchScratch&, const BatchTuning&,
                                              LaunchCfg&, bool);

}  // namespace lp
