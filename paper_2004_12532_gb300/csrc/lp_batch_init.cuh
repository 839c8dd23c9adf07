// lp_batch_init.cuh -- the batched engine's set-up of a launch (lp_batched.cu):
// each segment record's engine state and the launch's shared words.  The
// engine's own set-up kernel runs it; the quicksort runs it inside the kernel
// that builds a level's records, in place of that launch.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "lp_batched.h"
#include "lp_plan.h"

namespace lp {

enum : uint32_t { kSegOpen = 0, kSegDone = 2 };

// The engine state of a record whose caller's fields (keys, n, pivot, salt)
// are set: its 16-byte aligned body, level 0, open, and the seed of its
// offsets X -- from the batch seed and the segment's salt only, not from its
// place in the list.
template <typename T>
__device__ __forceinline__ void batch_seg_init(SegDesc& d, uint64_t batch_seed) {
  constexpr uint32_t K = sizeof(T), A = 16 / sizeof(T);
  const uintptr_t addr = reinterpret_cast<uintptr_t>(d.keys);
  uint64_t h = ((16 - (addr & 15)) & 15) / K;
  if (h > d.n) h = d.n;
  d.h = h;
  d.be = h + ((d.n - h) / A) * A;
  d.lo = h;
  d.hi = d.be;
  d.level = 0;
  d.state = kSegOpen;
  d.seed = sm_stream(batch_seed, d.salt);
  d.vmin = ~0ull;
  d.vmax = 0ull;
  d.count = 0ull;
  d.body_count = 0ull;
  d.t = 0ull;
}

// The launch's shared words, by threads i = 0 .. kBatchRoundSlots * 4 - 1 of
// the set-up: the streamed-key tally, the grid barrier (the status word is
// the caller's) and the round stamps start at zero.
__device__ __forceinline__ void batch_launch_reset(unsigned long long* traffic,
                                                   unsigned long long* tround, uint32_t* bar,
                                                   uint32_t i) {
  if (i == 0) {
    *traffic = 0ull;
    bar[0] = 0u;
    bar[1] = 0u;
  }
  if (i < kBatchRoundSlots * 4) tround[i] = 0ull;
}

}  // namespace lp
