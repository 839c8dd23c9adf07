// CPU emulation of the CTA-wide streaming group partition (stream_group in
// lp_smoothed.cuh), driven by the same control logic (lp_plan.h).  Data moves
// with plain copies; every hazard the GPU version must avoid is checked:
//   - a line is loaded once, and a stage is refilled only after consumption;
//   - a wait uses the parity of the load that filled the stage;
//   - a line is written once, and only after it was consumed;
//   - ring appends never overwrite ring bytes a pending bulk store still reads
//     (the kPendingFlushes most recent flushes are pending);
//   - the group ends partitioned, as a permutation, with k predecessors.
// Usage: emulate_stream <cases> <seed>; prints OK or the first failure.
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <deque>
#include <vector>

#include "lp_plan.h"

using namespace lp;

static uint64_t rs = 88172645463325252ull;
static uint64_t rnd() {
  rs ^= rs << 13; rs ^= rs >> 7; rs ^= rs << 17;
  return rs;
}

#define CHECK(c, ...)                         \
  do {                                        \
    if (!(c)) {                               \
      printf("FAIL line %d: ", __LINE__);     \
      printf(__VA_ARGS__);                    \
      printf("\n");                           \
      exit(1);                                \
    }                                         \
  } while (0)

struct Flush { int ring; uint64_t head, len; };

static bool overlaps(uint64_t a0, uint64_t alen, uint64_t b0, uint64_t blen, uint64_t ring) {
  // circular intervals [a0, a0+alen) and [b0, b0+blen) modulo ring
  if (alen == 0 || blen == 0) return false;
  return ((b0 - a0) % ring) < alen || ((a0 - b0) % ring) < blen;
}

// lines: nl lines of b keys, the last of length last_len; keys are 0/1 flags
// (1 = predecessor).
static void run_case(int64_t nl, uint64_t b, uint64_t last_len, int pattern, uint64_t ring_keys) {
  std::vector<std::vector<int>> line(nl);
  for (int64_t m = 0; m < nl; m++) {
    uint64_t len = (m == nl - 1) ? last_len : b;
    line[m].resize(len);
    for (uint64_t q = 0; q < len; q++) {
      int v;
      switch (pattern) {
        case 0: v = rnd() & 1; break;                       // 50%
        case 1: v = (rnd() % 100) == 0; break;              // 1% preds
        case 2: v = (rnd() % 100) != 0; break;              // 99% preds
        case 3: v = 1; break;                               // all preds
        case 4: v = 0; break;                               // all succs
        case 5: v = (m % 2) == 0; break;                    // alternating lines
        case 6: v = m < nl / 2; break;                      // sorted
        case 7: v = m >= nl / 2; break;                     // reverse sorted
        default: v = (rnd() % 7) < (uint64_t)(m % 8); break;
      }
      line[m][q] = v;
    }
  }
  std::vector<std::vector<int>> orig = line;
  uint64_t total = 0, preds = 0;
  for (auto& l : line) for (int v : l) { total++; preds += v; }

  std::vector<int> loaded(nl, 0), written(nl, 0);
  // stage state: which line it holds and the parity of the completion
  int64_t stage_line[kStages];
  int stage_busy[kStages];
  uint32_t stage_done_parity[kStages];
  uint32_t stage_completions[kStages];
  for (uint32_t s = 0; s < kStages; s++) {
    stage_line[s] = -1; stage_busy[s] = 0; stage_completions[s] = 0; stage_done_parity[s] = 0;
  }
  std::vector<int> stage_data[kStages];
  std::vector<int> pring(ring_keys), sring(ring_keys);
  std::deque<Flush> pending;

  StreamCtl c;
  ctl_init(c, nl);
  uint32_t phase = 0;

  auto issue = [&](int64_t m, uint32_t st) {
    CHECK(m >= 0 && m < nl, "issue out of range %lld", (long long)m);
    CHECK(!loaded[m], "line %lld loaded twice", (long long)m);
    CHECK(!stage_busy[st], "stage %u refilled before consumption", st);
    loaded[m] = 1;
    stage_busy[st] = 1;
    stage_line[st] = m;
    stage_data[st] = line[m];
    stage_done_parity[st] = stage_completions[st] & 1u;  // parity of this completion
    stage_completions[st]++;
  };
  auto do_flush = [&](int ring, uint64_t head, int64_t m) {
    CHECK(ctl_consumed(c, m), "flush into unconsumed line %lld", (long long)m);
    CHECK(!written[m], "line %lld written twice", (long long)m);
    written[m] = 1;
    std::vector<int>& r = ring ? sring : pring;
    for (uint64_t q = 0; q < line[m].size(); q++) line[m][q] = r[(head + q) % ring_keys];
    pending.push_back({ring, head, (uint64_t)line[m].size()});
  };

  for (uint32_t q = 0; q < kQ; q++) {
    if (ctl_can_issue(c)) { issue(c.fi, stage_front(c.fi)); c.fi++; }
    if (ctl_can_issue(c)) { issue(c.bi, stage_back(c, c.bi)); c.bi--; }
  }
  while (!ctl_done(c)) {
    const bool front = ctl_pick_front(c);
    const int64_t m = front ? c.lo_c : c.hi_c;
    const bool from_front_q = m < c.fi;
    const uint32_t st = ctl_stage_of(c, m);
    const uint64_t len = line[m].size();
    CHECK(ctl_p_count(c) + len + kPendingFlushes * b <= ring_keys, "P ring bound");
    CHECK(ctl_s_count(c) + len + kPendingFlushes * b <= ring_keys, "S ring bound");
    CHECK(stage_busy[st] && stage_line[st] == m, "stage %u does not hold line %lld", st,
          (long long)m);
    CHECK(((phase >> st) & 1u) == stage_done_parity[st], "parity mismatch at stage %u", st);
    // classify: append (checking pending regions)
    uint64_t np = 0;
    for (int v : stage_data[st]) np += v;
    for (auto& f : pending) {
      if (f.ring == 0)
        CHECK(!overlaps(c.p_tail, np, f.head, f.len, ring_keys), "P append over pending flush");
      else
        CHECK(!overlaps(c.s_tail, len - np, f.head, f.len, ring_keys),
              "S append over pending flush");
    }
    uint64_t pp = c.p_tail, sp = c.s_tail;
    for (int v : stage_data[st]) {
      if (v) pring[(pp++) % ring_keys] = v; else sring[(sp++) % ring_keys] = v;
    }
    phase ^= 1u << st;
    stage_busy[st] = 0;
    c.p_tail += np;
    c.s_tail += len - np;
    c.k += np;
    if (front) c.lo_c++; else c.hi_c--;
    if (ctl_can_issue(c)) {
      if (from_front_q) { issue(c.fi, stage_front(c.fi)); c.fi++; }
      else { issue(c.bi, stage_back(c, c.bi)); c.bi--; }
    }
    while (c.fw <= c.bw && ctl_consumed(c, c.fw)) {
      uint64_t lw = line[c.fw].size();
      if (ctl_p_count(c) < lw) break;
      do_flush(0, c.p_head, c.fw);
      c.p_head += lw;
      c.fw++;
    }
    while (c.bw >= c.fw && ctl_consumed(c, c.bw)) {
      uint64_t lw = line[c.bw].size();
      if (ctl_s_count(c) < lw) break;
      do_flush(1, c.s_head, c.bw);
      c.s_head += lw;
      c.bw--;
    }
    while (pending.size() > kPendingFlushes) pending.pop_front();
  }
  // remainder
  uint64_t pc = ctl_p_count(c), sc = ctl_s_count(c), rem = pc + sc;
  uint64_t cap = 0;
  for (int64_t m = c.fw; m <= c.bw; m++) {
    CHECK(!written[m], "remainder line %lld already written", (long long)m);
    cap += line[m].size();
  }
  CHECK(cap == rem, "remainder size %llu != capacity %llu", (unsigned long long)rem,
        (unsigned long long)cap);
  for (uint64_t q = 0; q < rem; q++) {
    int v = q < pc ? pring[(c.p_head + q) % ring_keys] : sring[(c.s_head + q - pc) % ring_keys];
    int64_t m = c.fw + (int64_t)(q / b);
    line[m][q % b] = v;
    written[m] = 1;
  }
  for (int64_t m = 0; m < nl; m++) CHECK(loaded[m] && written[m], "line %lld untouched", (long long)m);
  // partitioned, permutation (0/1 multiset), k
  CHECK(c.k == preds, "k %llu != preds %llu", (unsigned long long)c.k, (unsigned long long)preds);
  uint64_t pos = 0;
  for (auto& l : line)
    for (int v : l) {
      CHECK((pos < preds) == (v == 1), "not partitioned at slot %llu", (unsigned long long)pos);
      pos++;
    }
  (void)orig;
  (void)total;
}

int main(int argc, char** argv) {
  int cases = argc > 1 ? atoi(argv[1]) : 2000;
  rs ^= argc > 2 ? strtoull(argv[2], 0, 10) * 0x9E3779B97F4A7C15ull : 0;
  const uint64_t bs[] = {4, 8, 16, 64, 512};
  for (int t = 0; t < cases; t++) {
    uint64_t b = bs[rnd() % 5];
    int64_t nl = 1 + (int64_t)(rnd() % (t % 3 == 0 ? 300 : 24));
    uint64_t last = b;
    if (rnd() % 2) last = 1 + rnd() % b;
    int pattern = (int)(rnd() % 9);
    uint64_t ring = 8 * b;  // ring holds 8 full lines, as in the kernel
    run_case(nl, b, last, pattern, ring);
  }
  printf("OK\n");
  return 0;
}
