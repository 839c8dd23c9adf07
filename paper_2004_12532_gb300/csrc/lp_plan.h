// lp_plan.h -- pure integer planning logic shared by the CUDA kernels and
// their host code: step geometry, the per-level parameter rule, the random
// offsets X, and the control state of the CTA-wide streaming partition of one
// group.  Plain C++ with __host__ __device__ so the control logic can be
// exercised on the CPU as well.
//
// Notation follows Sec. 4 of Kuszmaul & Westover (arXiv 2004.12532):
// a step on a range of n keys uses lines of b keys; chunk j holds lines
// j*g .. j*g+g-1; group U_i holds line j*g + (X[j] + i) mod g of every chunk.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define LP_HD __host__ __device__ __forceinline__
#else
#define LP_HD inline
#endif

namespace lp {

// ---------------------------------------------------------------- constants
// The streaming kernels give one warp one group (the paper's "serial
// partition of U_i", one processor per group).  Per warp: kQ line loads in
// flight per side, two rings (P, S) of kRingLines lines, bulk stores allowed
// to read smem for up to kPendingFlushes write-backs.
constexpr uint32_t kLineBytesMax = 512;    // largest line (stage) in key bytes
constexpr uint32_t kLineBytesMin = 128;    // smallest line used by the parameter rule
constexpr uint32_t kQ = 4;                 // loads in flight per side (front / back)
constexpr uint32_t kStages = 2 * kQ;       // input stages per warp
constexpr uint32_t kRingLines = 8;         // ring capacity, in lines of the largest size
constexpr uint32_t kPendingFlushes = 2;    // bulk stores allowed to still read smem
constexpr uint32_t kLineTab = 16;          // issued-line table entries per side
constexpr uint32_t kBatchMax = 1;          // lines consumed per step
constexpr uint32_t kFinishBytes = 64 * 1024;  // ranges up to this size: one CTA in smem
constexpr uint32_t kMinChunks = 64;        // s at least this large when g > 1

// ------------------------------------------------------------ random source
// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): output k of the generator
// whose state starts at `seed`.
LP_HD uint64_t sm_stream(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

LP_HD uint64_t mulhi64(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// floor(r * g / 2^64): an offset in {0..g-1} from a uniform 64-bit word.
LP_HD uint64_t range_of(uint64_t r, uint64_t g) { return mulhi64(r, g); }

// Seed of the offsets X of level `level` of a run seeded with `seed`.
LP_HD uint64_t level_seed(uint64_t seed, uint64_t level) { return sm_stream(seed, level); }

// ------------------------------------------------------------ step geometry
struct StepGeom {
  uint64_t n;      // keys in the range
  uint64_t b;      // keys per line
  uint64_t g;      // groups (= lines per chunk)
  uint64_t L;      // lines, ceil(n / b); the last may be partial
  uint64_t s;      // chunks, ceil(L / g); lines >= L are virtual padding
  uint64_t sigma;  // level seed for X
  int strided;     // 1: X == 0 (the Strided Algorithm)
};

LP_HD StepGeom make_geom(uint64_t n, uint64_t b, uint64_t g, uint64_t sigma, int strided) {
  StepGeom G;
  G.n = n; G.b = b; G.g = g; G.sigma = sigma; G.strided = strided;
  G.L = (n + b - 1) / b;
  G.s = (G.L + g - 1) / g;
  return G;
}

// X[j], the random offset of chunk j.
LP_HD uint64_t offset_X(const StepGeom& G, uint64_t j) {
  return G.strided ? 0 : range_of(sm_stream(G.sigma, j), G.g);
}

// Line (within the range) holding the j-th line of group i.
LP_HD uint64_t group_line(const StepGeom& G, uint64_t i, uint64_t j) {
  uint64_t off = offset_X(G, j) + i;
  if (off >= G.g) off -= G.g;
  return j * G.g + off;
}

// Number of real lines of group i: s, minus one when its line of the last
// chunk is virtual.
LP_HD uint64_t group_num_lines(const StepGeom& G, uint64_t i) {
  if (G.s == 0) return 0;
  uint64_t last = group_line(G, i, G.s - 1);
  return last < G.L ? G.s : G.s - 1;
}

LP_HD uint64_t line_len(const StepGeom& G, uint64_t line) {
  uint64_t start = line * G.b;
  uint64_t end = start + G.b;
  return (end <= G.n ? end : G.n) - start;
}

// v_i (relative to the range start): the position of slot k of group i, or
// one past its last slot when k equals the group's size.  All lines of a
// group are full except possibly its last.
LP_HD uint64_t group_split_pos(const StepGeom& G, uint64_t i, uint64_t nl, uint64_t k) {
  uint64_t m = k / G.b;
  if (m >= nl) {
    uint64_t last = group_line(G, i, nl - 1);
    return last * G.b + line_len(G, last);
  }
  uint64_t line = group_line(G, i, m);
  uint64_t off = k - m * G.b;
  if (off >= line_len(G, line)) {  // k == size with the last line partial
    return line * G.b + line_len(G, line);
  }
  return line * G.b + off;
}

// ------------------------------------------------------------ parameter rule
// Chooses the line size b and the group count g of one step on n keys of
// key_bytes each, for `groups_max` concurrent group workers (warps) and lines
// of at most line_bytes_max bytes.  Large ranges get the largest line that
// still leaves at least kMinChunks chunks with one group per worker; smaller
// ranges get shorter lines, then fewer groups.  g == 0 means: at most
// finish_keys keys, which one CTA partitions in shared memory (the paper's
// base case).
struct StepParams { uint64_t b, g; };

LP_HD StepParams choose_params(uint64_t n, uint32_t key_bytes, uint64_t groups_max,
                               uint32_t line_bytes_max, uint64_t finish_keys) {
  StepParams P;
  P.b = line_bytes_max / key_bytes;
  P.g = 0;
  if (n <= finish_keys) return P;
  for (uint32_t lb = line_bytes_max; lb >= kLineBytesMin; lb >>= 1) {
    const uint64_t b = lb / key_bytes;
    const uint64_t g = n / (b * kMinChunks);
    P.b = b;
    P.g = g;
    if (g >= groups_max) { P.g = groups_max; return P; }
  }
  if (P.g < 2) P.g = 2;
  return P;
}

// ------------------------------------------------- streaming control state
// One CTA partitions one group as a stream of its nl lines (in group order):
// lines are loaded from both ends (kQ in flight per side), every consumed
// line's predecessors go to ring P and successors to ring S, and a full
// line's worth of P (S) is written back to the lowest (highest) unwritten
// line once that line has been consumed.  Each line is read once and written
// once; the last one or two lines take what is left in the rings, P first.
struct StreamCtl {
  int64_t nl;            // lines in the group
  int64_t fi, bi;        // next line to load from the front / the back
  int64_t lo_c, hi_c;    // lowest / highest line not yet consumed
  int64_t fw, bw;        // next line to receive P (front) / S (back)
  uint64_t p_head, p_tail, s_head, s_tail;  // ring counters, in keys
  uint64_t k;            // predecessors seen
};

LP_HD void ctl_init(StreamCtl& c, int64_t nl) {
  c.nl = nl; c.fi = 0; c.bi = nl - 1; c.lo_c = 0; c.hi_c = nl - 1;
  c.fw = 0; c.bw = nl - 1; c.p_head = c.p_tail = c.s_head = c.s_tail = 0; c.k = 0;
}
LP_HD bool ctl_can_issue(const StreamCtl& c) { return c.fi <= c.bi; }
LP_HD bool ctl_done(const StreamCtl& c) { return c.lo_c > c.hi_c; }
LP_HD uint32_t stage_front(int64_t line) { return (uint32_t)(line % kQ); }
LP_HD uint32_t stage_back(const StreamCtl& c, int64_t line) {
  return kQ + (uint32_t)((c.nl - 1 - line) % kQ);
}
// Stage holding an issued line: lines below fi came from the front.
LP_HD uint32_t ctl_stage_of(const StreamCtl& c, int64_t line) {
  return line < c.fi ? stage_front(line) : stage_back(c, line);
}
// Consume from the side whose written-behind slack is smaller (ties: front).
LP_HD bool ctl_pick_front(const StreamCtl& c) {
  return (c.lo_c - c.fw) <= (c.bw - c.hi_c);
}
LP_HD bool ctl_consumed(const StreamCtl& c, int64_t line) {
  return line < c.lo_c || line > c.hi_c;
}
LP_HD uint64_t ctl_p_count(const StreamCtl& c) { return c.p_tail - c.p_head; }
LP_HD uint64_t ctl_s_count(const StreamCtl& c) { return c.s_tail - c.s_head; }

// Picks up to maxw lines for the next batch with the slack policy, marking
// them consumed.  For each: the line, whether it was loaded from the front
// queue, and its stage.  Returns the number picked (0 once all are consumed).
LP_HD uint32_t ctl_pick_batch(StreamCtl& c, uint32_t maxw, int64_t* lines, bool* from_front,
                              uint32_t* stages) {
  uint32_t w = 0;
  while (w < maxw && !ctl_done(c)) {
    const bool front = ctl_pick_front(c);
    const int64_t line = front ? c.lo_c : c.hi_c;
    lines[w] = line;
    from_front[w] = line < c.fi;
    stages[w] = ctl_stage_of(c, line);
    if (front) c.lo_c++; else c.hi_c--;
    w++;
  }
  return w;
}

// Slot of a line in the per-CTA table of (line, length) records:
// front-issued lines in [0, kLineTab), back-issued in [kLineTab, 2 kLineTab).
LP_HD uint32_t line_tab_slot_side(const StreamCtl& c, int64_t line, bool front) {
  return front ? (uint32_t)(line % kLineTab)
               : kLineTab + (uint32_t)((c.nl - 1 - line) % kLineTab);
}
// Same for a line already issued (lines below fi came from the front).
LP_HD uint32_t line_tab_slot(const StreamCtl& c, int64_t line) {
  return line_tab_slot_side(c, line, line < c.fi);
}

}  // namespace lp
