// CPU emulation of the per-warp line-pair partition of one group
// (warp_pair_group in lp_smoothed.cuh), driven by the same control logic
// (PairCtl and the stage map of lp_plan.h).  Data moves with plain copies; the
// hazards the GPU version must avoid are checked:
//   - a line is loaded once; a stage is refilled only after it was taken;
//   - a take waits on the parity of the load that filled the stage;
//   - a line is written once, and only after it was taken;
//   - the group ends partitioned (predecessors first, in group order), as a
//     permutation of itself, with k predecessors.
// Usage: emulate_stream <cases> <seed>; prints OK or the first failure.
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
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

template <uint32_t Q>
static void run_case(int64_t nl, uint64_t b, uint64_t last_len, int pattern) {
  constexpr uint32_t kStages = 2 * Q;
  std::vector<std::vector<int64_t>> line(nl);
  int64_t id = 0;
  for (int64_t m = 0; m < nl; m++) {
    uint64_t len = (m == nl - 1) ? last_len : b;
    line[m].resize(len);
    for (uint64_t q = 0; q < len; q++) {
      int v;
      switch (pattern) {
        case 0: v = rnd() & 1; break;
        case 1: v = (rnd() % 100) == 0; break;
        case 2: v = (rnd() % 100) != 0; break;
        case 3: v = 1; break;
        case 4: v = 0; break;
        case 5: v = (m % 2) == 0; break;
        case 6: v = m < nl / 2; break;
        case 7: v = m >= nl / 2; break;
        default: v = (rnd() % 7) < (uint64_t)(m % 8); break;
      }
      line[m][q] = (id++) * 2 + v;  // low bit: predecessor flag
    }
  }
  std::vector<int64_t> all0;
  uint64_t preds = 0;
  for (auto& l : line)
    for (int64_t x : l) { all0.push_back(x); preds += x & 1; }

  std::vector<int> loaded(nl, 0), taken(nl, 0), written(nl, 0);
  int64_t stage_line[kStages];
  int stage_busy[kStages];
  uint32_t stage_parity[kStages], stage_uses[kStages];
  std::vector<int64_t> stage_data[kStages];
  for (uint32_t s = 0; s < kStages; s++) {
    stage_line[s] = -1; stage_busy[s] = 0; stage_parity[s] = 0; stage_uses[s] = 0;
  }
  PairCtl c;
  pair_init(c, nl);
  uint32_t phase = 0;
  uint64_t k = 0;

  auto issue = [&](int64_t m, uint32_t st) {
    CHECK(m >= 0 && m < nl, "issue out of range");
    CHECK(!loaded[m], "line %lld loaded twice", (long long)m);
    CHECK(!stage_busy[st], "stage %u refilled before it was taken", st);
    loaded[m] = 1;
    stage_busy[st] = 1;
    stage_line[st] = m;
    stage_data[st] = line[m];
    stage_parity[st] = stage_uses[st] & 1u;
    stage_uses[st]++;
  };
  auto take = [&](int64_t m, std::vector<int64_t>& reg) {
    const uint32_t st = pair_stage_of<Q>(c, m);
    const bool front_stage = st < Q;
    CHECK(stage_busy[st] && stage_line[st] == m, "stage %u does not hold line %lld", st,
          (long long)m);
    CHECK(((phase >> st) & 1u) == stage_parity[st], "parity mismatch");
    CHECK(!taken[m], "line taken twice");
    taken[m] = 1;
    phase ^= 1u << st;
    reg = stage_data[st];
    for (int64_t x : reg) k += x & 1;
    stage_busy[st] = 0;
    if (pair_can_issue(c)) {
      if (front_stage) {
        CHECK(pair_stage_front<Q>(c.fi) == st, "front refill into another stage");
        issue(c.fi, pair_stage_front<Q>(c.fi)); c.fi++;
      } else {
        CHECK(pair_stage_back<Q>(c, c.bi) == st, "back refill into another stage");
        issue(c.bi, pair_stage_back<Q>(c, c.bi)); c.bi--;
      }
    }
  };
  auto store = [&](int64_t m, const std::vector<int64_t>& reg) {
    CHECK(taken[m], "write before take");
    CHECK(!written[m], "line %lld written twice", (long long)m);
    written[m] = 1;
    line[m] = reg;
  };

  for (uint32_t q = 0; q < Q; q++) {
    if (pair_can_issue(c)) { issue(c.fi, pair_stage_front<Q>(c.fi)); c.fi++; }
    if (pair_can_issue(c)) { issue(c.bi, pair_stage_back<Q>(c, c.bi)); c.bi--; }
  }
  std::vector<int64_t> L, R;
  int64_t lL = -1, lR = -1;
  bool hasL = false, hasR = false;
  for (;;) {
    if (!hasL && pair_has_unread(c)) { lL = c.fnext; take(c.fnext, L); c.fnext++; hasL = true; }
    if (!hasR && pair_has_unread(c)) { lR = c.bnext; take(c.bnext, R); c.bnext--; hasR = true; }
    if (!(hasL && hasR)) break;
    std::vector<size_t> ls, rp;
    for (size_t q = 0; q < L.size(); q++) if (!(L[q] & 1)) ls.push_back(q);
    for (size_t q = 0; q < R.size(); q++) if (R[q] & 1) rp.push_back(q);
    const size_t m = std::min(ls.size(), rp.size());
    for (size_t j = 0; j < m; j++) std::swap(L[ls[j]], R[rp[j]]);
    const bool ln = ls.size() <= rp.size(), rn = rp.size() <= ls.size();
    if (ln) { store(lL, L); hasL = false; }
    if (rn) { store(lR, R); hasR = false; }
  }
  CHECK(c.fnext > c.bnext, "unread lines left");
  if (hasL || hasR) {
    std::vector<int64_t>& F = hasL ? L : R;
    std::stable_partition(F.begin(), F.end(), [](int64_t x) { return (x & 1) != 0; });
    store(hasL ? lL : lR, F);
  }
  for (int64_t m = 0; m < nl; m++)
    CHECK(loaded[m] && taken[m] && written[m], "line %lld untouched", (long long)m);
  CHECK(k == preds, "k %llu != preds %llu", (unsigned long long)k, (unsigned long long)preds);
  std::vector<int64_t> all1;
  uint64_t pos = 0;
  for (auto& l : line)
    for (int64_t x : l) {
      CHECK((pos < preds) == ((x & 1) != 0), "not partitioned at slot %llu",
            (unsigned long long)pos);
      all1.push_back(x);
      pos++;
    }
  std::sort(all0.begin(), all0.end());
  std::sort(all1.begin(), all1.end());
  CHECK(all0 == all1, "not a permutation");
}

int main(int argc, char** argv) {
  int cases = argc > 1 ? atoi(argv[1]) : 2000;
  rs ^= argc > 2 ? strtoull(argv[2], 0, 10) * 0x9E3779B97F4A7C15ull : 0;
  // lines of the kernel: up to 2048 key bytes, whole 16-byte vectors; both
  // queue depths the kernels use (2 lines per side for 2 KB lines, 4 for 1 KB)
  for (int t = 0; t < cases; t++) {
    const uint32_t kpv = (rnd() & 1) ? 2 : 4;          // keys per vector (u64 / u32)
    const uint32_t lv = 128u >> (rnd() % 5);            // vectors per line: 128..8
    const uint64_t b = (uint64_t)lv * kpv;
    const int64_t nl = 1 + (int64_t)(rnd() % (t % 3 == 0 ? 400 : 20));
    uint64_t last = b;
    if (rnd() % 2) last = kpv * (1 + rnd() % lv);
    if (t & 1) run_case<2>(nl, b, last, (int)(rnd() % 9));
    else run_case<4>(nl, b, last, (int)(rnd() % 9));
  }
  printf("OK\n");
  return 0;
}
