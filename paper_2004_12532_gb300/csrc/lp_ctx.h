// lp_ctx.h -- the library context (internal).  One context owns the
// scratch of the calls made on it; see include/libpartition.h.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/libpartition.h"
#include "lp_launch.h"

struct lp_ctx {
  int device = 0;
  uint32_t grid_u64 = 0, grid_u32 = 0, grid_kv = 0;
  uint32_t grid_batch_u64 = 0, grid_batch_u32 = 0;  // cooperative grids of the batched kernel
  void* d_scratch = nullptr;      // fixed scratch: descriptors, status, split
  size_t scratch_bytes = 0;
  uint64_t* h_pinned = nullptr;   // 64 bytes of pinned host memory for read-back
  uint64_t aux_bytes = 0;
  uint64_t last_launches = 0;
  std::string err;
  lp::TaskScratch task{};
  bool timing = false;
  bool events_made = false;
  bool last_timed = false;
  cudaEvent_t ev[3];             // around the kernels of a timed call
  cudaStream_t last_stream = nullptr;
  void* d_var = nullptr;         // per-call scratch of the low-space partition (grown)
  size_t var_bytes = 0;
  // batched partition: device segment records and plan space (grown), the
  // pinned staging buffer for uploads, and the tuning in force
  void* d_batch = nullptr;
  size_t batch_bytes = 0;
  void* h_batch = nullptr;
  size_t h_batch_bytes = 0;
  lp_batch_tuning tuning{0, 0, 0, 0, 0, 0};
  unsigned long long* last_batch_traffic = nullptr;  // streamed-keys counter of the last batch
  unsigned long long* last_batch_tround = nullptr;   // its round timestamps
  lp_sort_stats sort_stats{};                         // of the last quicksort
  unsigned long long* last_low_tl = nullptr;          // phase stamps of the last LP_LOWSPACE call
  uint32_t level_cap = 0;    // LP_SMOOTHED: level at which an open range is handed over (0: last)
  void* hostpart = nullptr;  // state of the host-array partition (lp_hostpart.cu)
};

namespace lp {
void hostpart_free(lp_ctx* c);
}


lp_status lp_fail(lp_ctx* c, lp_status s, const char* what);
// "device wait timed out" and the kinds of wait that gave up (status word bits).
const char* lp_timeout_what(uint32_t status);
lp_status lp_cuda_fail(lp_ctx* c, cudaError_t e, const char* where);
lp_status ensure_var(lp_ctx* c, size_t bytes, cudaStream_t stream);
lp_status ensure_events(lp_ctx* c);
