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
static void run_case(int64_t nl, uint64_t b, uint64_t last_len, int pattern, uint64_t ring_keys,
                     uint32_t maxw) {
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
  // issued-line table, as in the kernel: slot -> line (checks validity)
  std::vector<int64_t> tab(2 * kLineTab, -1);

  auto issue = [&](int64_t m, uint32_t st, bool front) {
    CHECK(m >= 0 && m < nl, "issue out of range %lld", (long long)m);
    CHECK(!loaded[m], "line %lld loaded twice", (long long)m);
    CHECK(!stage_busy[st], "stage %u refilled before consumption", st);
    loaded[m] = 1;
    stage_busy[st] = 1;
    stage_line[st] = m;
    stage_data[st] = line[m];
    stage_done_parity[st] = stage_completions[st] & 1u;  // parity of this completion
    stage_completions[st]++;
    tab[line_tab_slot_side(c, m, front)] = m;
  };
  auto tab_check = [&](int64_t m) {
    CHECK(tab[line_tab_slot(c, m)] == m, "line table slot of line %lld overwritten",
          (long long)m);
  };
  auto do_flush = [&](int ring, uint64_t head, int64_t m) {
    CHECK(ctl_consumed(c, m), "flush into unconsumed line %lld", (long long)m);
    CHECK(!written[m], "line %lld written twice", (long long)m);
    tab_check(m);
    written[m] = 1;
    std::vector<int>& r = ring ? sring : pring;
    for (uint64_t q = 0; q < line[m].size(); q++) line[m][q] = r[(head + q) % ring_keys];
    pending.push_back({ring, head, (uint64_t)line[m].size()});
  };

  for (uint32_t q = 0; q < kQ; q++) {
    if (ctl_can_issue(c)) { issue(c.fi, stage_front(c.fi), true); c.fi++; }
    if (ctl_can_issue(c)) { issue(c.bi, stage_back(c, c.bi), false); c.bi--; }
  }
  int64_t cur[kBatchMax];
  bool cur_ff[kBatchMax];
  uint32_t sts[kBatchMax];
  uint32_t n = ctl_pick_batch(c, maxw, cur, cur_ff, sts);
  uint32_t par[kBatchMax];
  for (uint32_t j = 0; j < n; j++) { par[j] = (phase >> sts[j]) & 1u; phase ^= 1u << sts[j]; }
  while (n > 0) {
    // workers: wait, classify, append in batch order
    uint64_t np_tot = 0, ns_tot = 0;
    for (uint32_t j = 0; j < n; j++) {
      const int64_t m = cur[j];
      const uint32_t st = sts[j];
      tab_check(m);
      CHECK(stage_busy[st] && stage_line[st] == m, "stage %u does not hold line %lld", st,
            (long long)m);
      CHECK(par[j] == stage_done_parity[st], "parity mismatch at stage %u", st);
      uint64_t np = 0;
      for (int v : stage_data[st]) np += v;
      uint64_t ns = stage_data[st].size() - np;
      for (auto& f : pending) {
        if (f.ring == 0)
          CHECK(!overlaps(c.p_tail + np_tot, np, f.head, f.len, ring_keys), "P append over pending");
        else
          CHECK(!overlaps(c.s_tail + ns_tot, ns, f.head, f.len, ring_keys), "S append over pending");
      }
      // the batch never overruns the unread part of its own ring
      CHECK(ctl_p_count(c) + np_tot + np <= ring_keys, "P ring overrun");
      CHECK(ctl_s_count(c) + ns_tot + ns <= ring_keys, "S ring overrun");
      uint64_t pp = c.p_tail + np_tot, sp = c.s_tail + ns_tot;
      for (int v : stage_data[st]) {
        if (v) pring[(pp++) % ring_keys] = v; else sring[(sp++) % ring_keys] = v;
      }
      np_tot += np;
      ns_tot += ns;
      stage_busy[st] = 0;
    }
    // thread 0: bookkeeping, refills, write-back plan, next batch
    c.p_tail += np_tot;
    c.s_tail += ns_tot;
    c.k += np_tot;
    for (uint32_t j = 0; j < n; j++) {
      if (!ctl_can_issue(c)) break;
      if (cur_ff[j]) { issue(c.fi, stage_front(c.fi), true); c.fi++; }
      else { issue(c.bi, stage_back(c, c.bi), false); c.bi--; }
    }
    while (c.fw <= c.bw && ctl_consumed(c, c.fw)) {
      tab_check(c.fw);
      uint64_t lw = line[c.fw].size();
      if (ctl_p_count(c) < lw) break;
      do_flush(0, c.p_head, c.fw);
      c.p_head += lw;
      c.fw++;
    }
    while (c.bw >= c.fw && ctl_consumed(c, c.bw)) {
      tab_check(c.bw);
      uint64_t lw = line[c.bw].size();
      if (ctl_s_count(c) < lw) break;
      do_flush(1, c.s_head, c.bw);
      c.s_head += lw;
      c.bw--;
    }
    const uint64_t need = (uint64_t)(maxw + kPendingFlushes) * b;
    CHECK(ctl_p_count(c) + need <= ring_keys, "P ring bound (kernel check would abort)");
    CHECK(ctl_s_count(c) + need <= ring_keys, "S ring bound (kernel check would abort)");
    n = ctl_pick_batch(c, maxw, cur, cur_ff, sts);
    for (uint32_t j = 0; j < n; j++) { par[j] = (phase >> sts[j]) & 1u; phase ^= 1u << sts[j]; }
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
    tab_check(m);
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
  // line sizes in 16-byte vectors, as the kernel maps them: 2048-byte lines
  // (the largest) down to 512-byte lines; keys per vector 2 (u64) or 4 (u32)
  // per-warp geometry of the kernel: the largest line is 512 key bytes (32
  // vectors); levels use lines down to 128 bytes (8 vectors); rings hold 8
  // lines of the largest size; one line per step.
  for (int t = 0; t < cases; t++) {
    const uint32_t max_lv = 32;
    uint32_t lv = max_lv >> (rnd() % 3);
    uint32_t kpv = (rnd() & 1) ? 2 : 4;
    uint64_t b = (uint64_t)lv * kpv;
    int64_t nl = 1 + (int64_t)(rnd() % (t % 3 == 0 ? 400 : 30));
    uint64_t last = b;
    if (rnd() % 2) last = kpv * (1 + rnd() % lv);  // partial last line, whole vectors
    int pattern = (int)(rnd() % 9);
    uint64_t ring = (uint64_t)kRingLines * max_lv * kpv;
    run_case(nl, b, last, pattern, ring, kBatchMax);
  }
  printf("OK\n");
  return 0;
}
