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
// The streaming kernels give a group to one warp at a time (the paper's
// "serial partition of U_i", one processor per group).  A warp holds two
// lines of its group in registers (the paper's `low` and `high` ends) and
// keeps Q more lines in flight per side in shared memory.
constexpr uint32_t kLineBytesMax = 2048;   // largest line in key bytes (over all key types)
// largest line of a key type: 2 KB (fewer, longer line pairs per key; the
// kernels cap their registers so that two CTAs share an SM)
LP_HD constexpr uint32_t max_line_bytes(uint32_t key_bytes) {
  return key_bytes == 8 || key_bytes == 4 ? 2048u : 1024u;
}
constexpr uint32_t kLineBytesMin = 128;    // smallest line used by the parameter rule
constexpr uint32_t kFinishBytes = 64 * 1024;  // ranges up to this size: one CTA in smem
constexpr uint32_t kMinChunks = 8;         // lines per group, at least (when g > 1)

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
// Line size b and group count g of one step on n keys of key_bytes each: the
// largest line, at most `workers` groups (the callers pass the warp count, or
// a multiple of it when warps take several groups), but at least min_chunks
// chunks (lines per group).  Each level then shrinks
// the open range by roughly s / 3 at least; a range the CTAs can hold on chip
// is finished there instead (the paper's base case).
struct StepParams { uint64_t b, g; };

LP_HD StepParams choose_params(uint64_t n, uint32_t key_bytes, uint64_t workers,
                               uint32_t line_bytes, uint32_t min_chunks = kMinChunks) {
  StepParams P;
  P.b = line_bytes / key_bytes;
  P.g = n / (P.b * (min_chunks ? min_chunks : 1));
  if (P.g > workers) P.g = workers;
  if (P.g < 1) P.g = 1;
  return P;
}

// --------------------------------------------- line-pair (Hoare) control
// A warp partitions its group as the paper's serial two-pointer scan does,
// one line at a time instead of one key: it holds the lowest unfinished line
// L and the highest unfinished line R, swaps the j-th successor of L with the
// j-th predecessor of R for j < min(#succ(L), #pred(R)), and writes back
// whichever line became pure (L all predecessors, or R all successors; both
// when the counts match), then takes the next line from that side.  When no
// unread line is left, the line still in hand is partitioned on its own.
// Lines are loaded ahead from both ends, Q per side (Q a power of two; stages
// 0..Q-1 hold front lines, Q..2Q-1 back lines); `fi` / `bi` are the next lines
// to load from the front / back, [fnext, bnext] the lines not yet taken.
struct PairCtl {
  int32_t nl;            // lines in the group
  int32_t fi, bi;        // next line to load from the front / the back
  int32_t fnext, bnext;  // lines not yet taken: [fnext, bnext]
};

LP_HD void pair_init(PairCtl& c, int32_t nl) {
  c.nl = nl; c.fi = 0; c.bi = nl - 1; c.fnext = 0; c.bnext = nl - 1;
}
LP_HD bool pair_can_issue(const PairCtl& c) { return c.fi <= c.bi; }
template <uint32_t Q>
LP_HD uint32_t pair_stage_front(int32_t line) { return (uint32_t)line & (Q - 1); }
template <uint32_t Q>
LP_HD uint32_t pair_stage_back(const PairCtl& c, int32_t line) {
  return Q + ((uint32_t)(c.nl - 1 - line) & (Q - 1));
}
// Stage holding an issued line: lines below fi came from the front queue.
template <uint32_t Q>
LP_HD uint32_t pair_stage_of(const PairCtl& c, int32_t line) {
  return line < c.fi ? pair_stage_front<Q>(line) : pair_stage_back<Q>(c, line);
}
LP_HD bool pair_has_unread(const PairCtl& c) { return c.fnext <= c.bnext; }

}  // namespace lp
