// CPU test of the host-array partition plan (csrc/lp_hostpart.h): the
// library's own header, driven the way the library drives it, with the
// device replaced by a second array and the device partition by a serial one.
// A chunk is copied to the "device" only when it is partitioned (the latest
// moment a real upload can complete), so a copy back that came too early
// would corrupt a later chunk's input.  Checks: every plan finishes; the host
// array ends partitioned with the right split and the same multiset; the
// result does not depend on how far ahead the uploads run.
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <random>
#include <vector>

#include "lp_hostpart.h"

using lp::HostChunkPlan;
using lp::HostPiece;

static bool run(std::vector<uint64_t>& host, uint64_t pivot, uint64_t C, uint32_t lag,
                uint32_t ahead, uint64_t* split) {
  const uint64_t n = host.size();
  std::vector<uint64_t> dev(n, 0xdeadbeefull);
  HostChunkPlan plan;
  plan.init(n, C, lag);
  std::vector<HostPiece> pieces;
  std::vector<uint32_t> queue;  // uploaded, not yet partitioned
  size_t qh = 0;
  uint64_t guard = 0;
  while (!plan.finished()) {
    if (++guard > 10 * (uint64_t)plan.chunks() + 100) return false;
    // issue uploads as far ahead as allowed (at most `ahead` unprocessed)
    while (plan.uploads() < plan.chunks() && plan.processed() >= plan.needed_for_next() &&
           plan.uploads() - plan.processed() < ahead)
      queue.push_back(plan.next_upload());
    if (qh < queue.size()) {
      const uint32_t k = queue[qh++];
      const uint64_t b = plan.chunk_begin(k), len = plan.chunk_len(k);
      std::copy(host.begin() + b, host.begin() + b + len, dev.begin() + b);  // the upload lands
      const auto mid = std::stable_partition(dev.begin() + b, dev.begin() + b + len,
                                             [&](uint64_t x) { return x <= pivot; });
      if (!plan.partitioned((uint64_t)(mid - (dev.begin() + b)))) return false;
    } else if (plan.processed() < plan.needed_for_next()) {
      return false;  // nothing in flight, yet the next choice waits for a count
    }
    pieces.clear();
    plan.take_pieces(pieces);
    for (const HostPiece& p : pieces)
      std::copy(dev.begin() + p.dev, dev.begin() + p.dev + p.len, host.begin() + p.host);
  }
  *split = plan.split();
  return true;
}

static int check(const std::vector<uint64_t>& in, uint64_t pivot, uint64_t C, uint32_t lag,
                 const char* what) {
  std::vector<uint64_t> ref;
  for (int ahead : {1, 2, 3, 8, 1000}) {
    if ((uint32_t)ahead < lag) continue;  // the library keeps at least `lag` uploads ahead
    std::vector<uint64_t> h = in;
    uint64_t t = 0;
    if (!run(h, pivot, C, lag, (uint32_t)ahead, &t)) {
      printf("FAIL %s: plan stuck (n=%zu C=%llu lag=%u ahead=%d)\n", what, in.size(),
             (unsigned long long)C, lag, ahead);
      return 1;
    }
    const uint64_t want = (uint64_t)std::count_if(in.begin(), in.end(),
                                                  [&](uint64_t x) { return x <= pivot; });
    if (t != want) { printf("FAIL %s: split %llu want %llu\n", what, (unsigned long long)t, (unsigned long long)want); return 1; }
    for (uint64_t i = 0; i < h.size(); i++)
      if ((h[i] <= pivot) != (i < t)) { printf("FAIL %s: not partitioned at %llu\n", what, (unsigned long long)i); return 1; }
    std::vector<uint64_t> a = in, b = h;
    std::sort(a.begin(), a.end());
    std::sort(b.begin(), b.end());
    if (a != b) { printf("FAIL %s: multiset changed (ahead=%d)\n", what, ahead); return 1; }
    if (ref.empty()) ref = h;
    else if (ref != h) { printf("FAIL %s: result depends on ahead=%d\n", what, ahead); return 1; }
  }
  return 0;
}

int main(int argc, char** argv) {
  const int trials = argc > 1 ? atoi(argv[1]) : 300;
  std::mt19937_64 rng(12345);
  int bad = 0;
  for (int tr = 0; tr < trials && !bad; tr++) {
    const uint64_t n = 1 + rng() % 5000;
    const uint64_t C = 1 + rng() % 700;
    const uint32_t lag = 1 + (uint32_t)(rng() % 4);
    std::vector<uint64_t> in(n);
    const int kind = (int)(rng() % 7);
    for (uint64_t i = 0; i < n; i++) in[i] = rng() % 1000;
    uint64_t pivot = rng() % 1000;
    if (kind == 1) pivot = 1000;          // all predecessors
    if (kind == 2) pivot = 0, std::fill(in.begin(), in.end(), 5);  // all successors
    if (kind == 3) std::sort(in.begin(), in.end());                 // predecessors in front
    if (kind == 4) std::sort(in.rbegin(), in.rend());               // ... at the back
    if (kind == 5)  // blocks alternating between all-predecessor and all-successor
      for (uint64_t i = 0; i < n; i++) in[i] = ((i / (1 + C / 2)) & 1) ? 999 : 0, pivot = 500;
    if (kind == 6) for (uint64_t i = 0; i < n; i++) in[i] = (i * 7919) % 1000;
    bad |= check(in, pivot, C, lag, "random");
  }
  // a split larger than its chunk is refused and plans nothing; the plan then
  // accepts the chunk's real split
  if (!bad) {
    HostChunkPlan plan;
    plan.init(1000, 300, 2);
    const uint32_t k = plan.next_upload();
    const uint64_t len = plan.chunk_len(k);
    std::vector<HostPiece> pieces;
    if (plan.partitioned(len + 1) || plan.processed() != 0) {
      printf("FAIL: a split above the chunk length was accepted\n");
      bad = 1;
    }
    plan.take_pieces(pieces);
    if (!bad && !pieces.empty()) {
      printf("FAIL: copies planned from a refused split\n");
      bad = 1;
    }
    if (!bad && (!plan.partitioned(len / 2) || plan.processed() != 1)) {
      printf("FAIL: a valid split after a refused one\n");
      bad = 1;
    }
  }
  if (!bad) printf("OK\n");
  return bad;
}
