// Host checks of the serving engine's arena and admission rule (lp_sched.h):
// random allocation / release sequences against a byte-level shadow map, and
// FIFO admission under a slot limit and a budget.  Prints OK or the failure.
#include <stdio.h>
#include <stdlib.h>

#include <deque>
#include <map>
#include <vector>

#include "lp_sched.h"

static unsigned long long rng_state = 1;
static unsigned long long rnd() {  // SplitMix64
  unsigned long long z = (rng_state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

#define CHECK(c, ...)                                         \
  do {                                                        \
    if (!(c)) {                                               \
      printf("FAIL line %d: ", __LINE__);                     \
      printf(__VA_ARGS__);                                    \
      printf("\n");                                           \
      return 1;                                               \
    }                                                         \
  } while (0)

static int arena_random(unsigned long long seed, int ops) {
  rng_state = seed;
  const uint64_t cap = 1 << 20;
  lp::Arena A(cap);
  std::map<uint64_t, uint64_t> live;  // offset -> rounded size
  std::vector<unsigned char> owner(cap, 0);
  for (int op = 0; op < ops; op++) {
    const bool do_alloc = live.empty() || (rnd() % 100) < 55;
    if (do_alloc) {
      const uint64_t want = 1 + rnd() % (cap / 16);
      uint64_t off = 0;
      const uint64_t largest = A.largest_free();
      const bool ok = A.alloc(want, &off);
      const uint64_t need = lp::Arena::rounded(want);
      CHECK(ok == (need <= largest), "alloc %llu: ok=%d largest=%llu", (unsigned long long)want,
            ok, (unsigned long long)largest);
      if (!ok) continue;
      CHECK(off % lp::Arena::kArenaAlign == 0, "misaligned offset");
      CHECK(off + need <= cap, "block past the end");
      for (uint64_t b = off; b < off + need; b++) {
        CHECK(!owner[b], "overlap at byte %llu", (unsigned long long)b);
        owner[b] = 1;
      }
      live[off] = need;
    } else {
      auto it = live.begin();
      std::advance(it, rnd() % live.size());
      CHECK(A.release(it->first), "release of a live block refused");
      for (uint64_t b = it->first; b < it->first + it->second; b++) owner[b] = 0;
      live.erase(it);
    }
    uint64_t used = 0;
    for (auto& kv : live) used += kv.second;
    CHECK(A.used() == used, "used %llu != %llu", (unsigned long long)A.used(),
          (unsigned long long)used);
    CHECK(A.live_blocks() == live.size(), "live count");
  }
  CHECK(!A.release(12345), "release of a non-block accepted");
  for (auto& kv : live) A.release(kv.first);
  CHECK(A.used() == 0 && A.free_runs() == 1 && A.largest_free() == cap,
        "frees did not coalesce: runs=%llu", (unsigned long long)A.free_runs());
  return 0;
}

static int admission() {
  // requests of given sizes; budget 1000 (after rounding to 256: units of 256)
  lp::Arena A(1024 * 4);
  std::deque<uint64_t> q;
  std::vector<uint64_t> size = {1000, 3000, 100, 5000, 200};
  for (uint64_t i = 0; i < size.size(); i++) q.push_back(i);
  std::map<uint64_t, uint64_t> offs;
  auto fits = [&](uint64_t id) {
    uint64_t off;
    if (!A.alloc(size[id], &off)) return false;
    offs[id] = off;
    return true;
  };
  uint64_t adm[8];
  // two slots: 0 and 1 fit (1024 + 3072 = 4096)
  uint32_t k = lp::admit_fifo(q, 2, fits, adm, 8);
  CHECK(k == 2 && adm[0] == 0 && adm[1] == 1, "first admission k=%u", k);
  // slots free but no budget: 2 (256 bytes) must wait, nothing overtakes it
  k = lp::admit_fifo(q, 3, fits, adm, 8);
  CHECK(k == 0 && q.front() == 2, "admitted without budget");
  A.release(offs[0]);
  k = lp::admit_fifo(q, 3, fits, adm, 8);
  // 2 fits (256), 3 (5000) never fits the budget: it blocks 4
  CHECK(k == 1 && adm[0] == 2 && q.front() == 3, "second admission k=%u", k);
  k = lp::admit_fifo(q, 0, fits, adm, 8);
  CHECK(k == 0, "admitted without a slot");
  return 0;
}

int main(int argc, char** argv) {
  const int ops = argc > 1 ? atoi(argv[1]) : 20000;
  for (unsigned long long s = 1; s <= 4; s++)
    if (arena_random(s, ops)) return 1;
  if (admission()) return 1;
  printf("OK\n");
  return 0;
}
