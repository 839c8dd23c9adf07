// lp_api.cu -- the C ABI of libpartition (include/libpartition.h): argument
// checks, context and scratch ownership, status mapping.  Every compute step
// runs in the kernels of lp_kernels.cu and its siblings.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>

#include "../../include/libpartition.h"
#include "lp_batched.h"
#include "lp_ctx.h"
#include "lp_qs.cuh"
#include "lp_device.cuh"
#include "lp_launch.h"
#include "lp_plan.h"
#include "lp_trace.h"

const char* lp_timeout_what(uint32_t st) {
  static thread_local char msg[160];
  static const struct { uint32_t bit; const char* name; } sites[] = {
      {lp::kSitePartition, "partition barrier"}, {lp::kSiteLowspace, "low-space barrier"},
      {lp::kSiteRounds, "engine round barrier"},  {lp::kSiteSortLoop, "sort level barrier"},
      {lp::kSiteLine, "line copy"},               {lp::kSiteBulk, "range copy"}};
  int o = snprintf(msg, sizeof(msg), "device wait timed out");
  const char* sep = " (";
  for (const auto& x : sites) {
    if ((st & x.bit) && o > 0 && o < (int)sizeof(msg)) {
      o += snprintf(msg + o, sizeof(msg) - o, "%s%s", sep, x.name);
      sep = ", ";
    }
  }
  if (sep[0] == ',' && o > 0 && o < (int)sizeof(msg)) snprintf(msg + o, sizeof(msg) - o, ")");
  return msg;
}

lp_status lp_fail(lp_ctx* c, lp_status s, const char* what) {
  if (c) c->err = what;
  return s;
}

lp_status lp_cuda_fail(lp_ctx* c, cudaError_t e, const char* where) {
  if (c) {
    c->err = std::string(where) + ": " + cudaGetErrorString(e);
  }
  return LP_ERR_CUDA;
}

namespace {

inline lp_status fail(lp_ctx* c, lp_status s, const char* what) { return lp_fail(c, s, what); }
inline lp_status cuda_fail(lp_ctx* c, cudaError_t e, const char* where) {
  return lp_cuda_fail(c, e, where);
}

lp_status status_to_lp(lp_ctx* c, uint32_t st) {
  if (st == 0) return LP_OK;
  if (st & lp::kStatTimeout) return fail(c, LP_ERR_TIMEOUT, lp_timeout_what(st));
  return fail(c, LP_ERR_INTERNAL, "device consistency check failed");
}

template <typename T>
bool aligned_to(const T* p, uintptr_t a) {
  return (reinterpret_cast<uintptr_t>(p) % a) == 0;
}

// Synchronous tail shared by the sync partition calls: read back split and
// status words.
lp_status read_back(lp_ctx* c, cudaStream_t stream, uint64_t* split_out) {
  cudaError_t e = cudaMemcpyAsync(c->h_pinned, c->task.split, 8, cudaMemcpyDeviceToHost, stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "read split");
  e = cudaMemcpyAsync(c->h_pinned + 1, c->task.status, 4, cudaMemcpyDeviceToHost, stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "read status");
  e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
  uint32_t st = (uint32_t)(c->h_pinned[1] & 0xffffffffu);
  if (split_out) *split_out = c->h_pinned[0];
  return status_to_lp(c, st);
}

}  // namespace

// Grows the context's per-call scratch to at least `bytes` (a stream-ordered
// free of the old buffer is not needed: the stream is synchronised first).
lp_status ensure_var(lp_ctx* c, size_t bytes, cudaStream_t stream) {
  if (bytes <= c->var_bytes) return LP_OK;
  cudaError_t e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
  if (c->d_var) cudaFree(c->d_var);
  c->d_var = nullptr;
  c->var_bytes = 0;
  e = cudaMalloc(&c->d_var, bytes);
  if (e != cudaSuccess) return fail(c, LP_ERR_OOM, "scratch allocation failed");
  c->var_bytes = bytes;
  c->aux_bytes = c->scratch_bytes + c->var_bytes + c->batch_bytes;
  return LP_OK;
}

// Creates the context's timing events once.
lp_status ensure_events(lp_ctx* c) {
  if (c->events_made) return LP_OK;
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  for (int i = 0; i < 3; i++) {
    e = cudaEventCreate(&c->ev[i]);
    if (e != cudaSuccess) {
      for (int j = 0; j < i; j++) cudaEventDestroy(c->ev[j]);
      return cuda_fail(c, e, "cudaEventCreate");
    }
  }
  c->events_made = true;
  return LP_OK;
}

namespace {

constexpr uint64_t kLowspaceBlock = 4096;  // B of the low-space partition (Sec. 5)

template <typename T, bool KV>
lp_status partition_impl(lp_ctx* c, T* keys, uint64_t* vals, uint64_t n, T pivot,
                         lp_variant variant, uint64_t seed, cudaStream_t stream,
                         uint64_t* split_out, uint64_t* d_split) {
  if (!c) return LP_ERR_INVALID_ARG;
  c->err.clear();
  c->last_launches = 0;
  c->last_low_tl = nullptr;
  if (variant != LP_SMOOTHED && variant != LP_STRIDED && variant != LP_LOWSPACE &&
      variant != LP_HYBRID)
    return fail(c, LP_ERR_INVALID_ARG, "unknown variant");
  if (n > 0 && (!keys || (KV && !vals))) return fail(c, LP_ERR_INVALID_ARG, "null array");
  if (!aligned_to(keys, sizeof(T)) || (KV && !aligned_to(vals, 8)))
    return fail(c, LP_ERR_INVALID_ARG, "array not naturally aligned");
  if (KV && n > lp::small_limit(sizeof(T), true) &&
      (reinterpret_cast<uintptr_t>(keys) & 15) != (reinterpret_cast<uintptr_t>(vals) & 15))
    return fail(c, LP_ERR_MISALIGNED, "keys and vals must share their offset mod 16");
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  lp::TaskScratch S = c->task;
  if (d_split) S.split = d_split;
  if (n == 0) {
    if (d_split) {
      e = cudaMemsetAsync(d_split, 0, 8, stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "memset split");
    }
    if (split_out) *split_out = 0;
    return LP_OK;
  }
  lp::LaunchCfg cfg{KV ? c->grid_kv : (sizeof(T) == 8 ? c->grid_u64 : c->grid_u32), stream, 0,
                    c->timing ? c->ev : nullptr};
  c->last_timed = c->timing;
  c->last_stream = stream;
  const bool small = n <= lp::small_limit(sizeof(T), KV);
  if (variant == LP_SMOOTHED || small) {
    // scratch for the residual-shrink guard's low-space handoff, when the
    // array is too large to finish on chip at level 0
    void* hv = nullptr;
    if (!small && lp::smoothed_may_hand_off<T, KV>(n, cfg.grid)) {
      lp_status ls =
          ensure_var(c, lp::lowspace_scratch_bytes(n, lp::kHandoffBlock, cfg.grid), stream);
      if (ls != LP_OK) return ls;
      hv = c->d_var;
    }
    e = lp::launch_smoothed<T, KV>(keys, vals, n, pivot, seed, 0, S, cfg, hv, c->level_cap);
  } else if (variant == LP_LOWSPACE) {
    lp_status ls = ensure_var(c, lp::lowspace_scratch_bytes(n, kLowspaceBlock, cfg.grid), stream);
    if (ls != LP_OK) return ls;
    cfg.phase_stamps = &c->last_low_tl;
    e = cudaSuccess;
    // the status word and grid barrier start clean
    e = cudaMemsetAsync(S.status, 0, 4, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(S.bar, 0, 8, stream);
    if (cfg.events && e == cudaSuccess) e = cudaEventRecord(cfg.events[0], stream);
    if (e == cudaSuccess)
      e = lp::launch_lowspace<T, KV>(keys, vals, 0, n, n, nullptr, pivot, kLowspaceBlock, ~0ull,
                                     c->d_var, S, S.split, cfg);
    if (cfg.events && e == cudaSuccess) e = cudaEventRecord(cfg.events[1], stream);
  } else {
    // Strided (X == 0) or Hybrid (random X): one Partial Partition Step, then
    // the open range [v_min, v_max) by the low-space partition
    lp_status ls = ensure_var(c, lp::lowspace_scratch_bytes(n, kLowspaceBlock, cfg.grid), stream);
    if (ls != LP_OK) return ls;
    uint64_t h = 0, body_end = 0;
    cudaEvent_t* evs = cfg.events;
    cfg.events = nullptr;
    if (evs) cudaEventRecord(evs[0], stream);
    e = lp::launch_first_level<T, KV>(keys, vals, n, pivot, seed, variant == LP_STRIDED ? 1 : 0,
                                      S, cfg, &h, &body_end);
    if (e == cudaSuccess)
      e = lp::launch_lowspace<T, KV>(keys, vals, 0, 0, n, S.desc, pivot, kLowspaceBlock, ~0ull,
                                     c->d_var, S, nullptr, cfg);
    if (evs && e == cudaSuccess) e = cudaEventRecord(evs[1], stream);
    if (e == cudaSuccess) e = lp::launch_finalize<T, KV>(keys, vals, n, h, body_end, pivot, S, cfg);
    cfg.events = evs;
  }
  c->last_launches = cfg.launches;
  if (e != cudaSuccess) return cuda_fail(c, e, "launch");
  if (split_out) {
    if (d_split) {
      e = cudaMemcpyAsync(c->h_pinned, d_split, 8, cudaMemcpyDeviceToHost, stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "read split");
      e = cudaMemcpyAsync(c->h_pinned + 1, c->task.status, 4, cudaMemcpyDeviceToHost, stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "read status");
      e = cudaStreamSynchronize(stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
      *split_out = c->h_pinned[0];
      return status_to_lp(c, (uint32_t)c->h_pinned[1]);
    }
    return read_back(c, stream, split_out);
  }
  return LP_OK;
}

template <typename T>
lp_status step_impl(lp_ctx* c, T* keys, uint64_t n, T pivot, uint64_t b, uint64_t g,
                    uint64_t seed, uint64_t level, int strided, cudaStream_t stream,
                    uint64_t* vmin, uint64_t* vmax, uint64_t* count) {
  if (!c) return LP_ERR_INVALID_ARG;
  c->err.clear();
  c->last_launches = 0;
  if (!vmin || !vmax || !count) return fail(c, LP_ERR_INVALID_ARG, "null result pointer");
  if (n > 0 && !keys) return fail(c, LP_ERR_INVALID_ARG, "null array");
  if (b == 0 || g == 0) return fail(c, LP_ERR_INVALID_ARG, "b and g must be positive");
  if ((b * sizeof(T)) % 16 != 0 || b * sizeof(T) > lp::max_line_bytes(sizeof(T)))
    return fail(c, LP_ERR_INVALID_ARG, "b*sizeof(key) must be a multiple of 16, at most 1024");
  if (!aligned_to(keys, 16) || (n * sizeof(T)) % 16 != 0)
    return fail(c, LP_ERR_MISALIGNED, "keys must be 16-byte aligned, n*sizeof(key) % 16 == 0");
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  if (n == 0) {
    *vmin = *vmax = *count = 0;
    return LP_OK;
  }
  lp::LaunchCfg cfg{sizeof(T) == 8 ? c->grid_u64 : c->grid_u32, stream, 0, nullptr};
  c->last_timed = false;
  c->last_stream = stream;
  e = lp::launch_step<T>(keys, n, pivot, b, g, seed, level, strided, c->task, cfg);
  c->last_launches = cfg.launches;
  if (e != cudaSuccess) return cuda_fail(c, e, "launch");
  // descriptor 0: vmin, vmax, count are its first three words
  e = cudaMemcpyAsync(c->h_pinned, c->task.desc, 24, cudaMemcpyDeviceToHost, stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "read result");
  e = cudaMemcpyAsync(c->h_pinned + 3, c->task.status, 4, cudaMemcpyDeviceToHost, stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "read status");
  e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
  uint64_t lo = c->h_pinned[0], hi = c->h_pinned[1];
  if (lo == ~0ull) lo = hi = 0;  // every group empty
  *vmin = lo;
  *vmax = hi;
  *count = c->h_pinned[2];
  return status_to_lp(c, (uint32_t)c->h_pinned[3]);
}

template <typename T>
lp_status lowspace_impl(lp_ctx* c, T* keys, uint64_t n, T pivot, uint64_t B, uint64_t base_keys,
                        cudaStream_t stream, uint64_t* split_out) {
  if (!c) return LP_ERR_INVALID_ARG;
  c->err.clear();
  c->last_launches = 0;
  if (!split_out) return fail(c, LP_ERR_INVALID_ARG, "null split_out");
  if (n > 0 && !keys) return fail(c, LP_ERR_INVALID_ARG, "null array");
  if (B == 0) return fail(c, LP_ERR_INVALID_ARG, "block size must be positive");
  if (!aligned_to(keys, sizeof(T))) return fail(c, LP_ERR_INVALID_ARG, "array not aligned");
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  if (n == 0) { *split_out = 0; return LP_OK; }
  lp::LaunchCfg cfg{sizeof(T) == 8 ? c->grid_u64 : c->grid_u32, stream, 0, nullptr};
  c->last_timed = false;
  c->last_stream = stream;
  lp_status ls = ensure_var(c, lp::lowspace_scratch_bytes(n, B, cfg.grid), stream);
  if (ls != LP_OK) return ls;
  lp::TaskScratch S = c->task;
  c->last_low_tl = nullptr;
  cfg.phase_stamps = &c->last_low_tl;
  e = cudaMemsetAsync(S.status, 0, 4, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(S.bar, 0, 8, stream);
  if (e == cudaSuccess)
    e = lp::launch_lowspace<T, false>(keys, nullptr, 0, n, n, nullptr, pivot, B,
                                      base_keys ? base_keys : 1, c->d_var, S, S.split, cfg);
  c->last_launches = cfg.launches;
  if (e != cudaSuccess) return cuda_fail(c, e, "launch");
  return read_back(c, stream, split_out);
}

template <typename T>
lp_status implicit_impl(lp_ctx* c, T* keys, uint64_t n, T pivot, uint64_t B, uint64_t base_keys,
                        int prefix_only, cudaStream_t stream, uint64_t* split_out) {
  if (!c) return LP_ERR_INVALID_ARG;
  c->err.clear();
  c->last_launches = 0;
  if (!split_out) return fail(c, LP_ERR_INVALID_ARG, "null split_out");
  if (n > 0 && !keys) return fail(c, LP_ERR_INVALID_ARG, "null array");
  if (!aligned_to(keys, sizeof(T))) return fail(c, LP_ERR_INVALID_ARG, "array not aligned");
  const uint32_t L = lp::lowspace_value_bits(n);
  if (L > lp::lowspace_value_bits_max())
    return fail(c, LP_ERR_INVALID_ARG, "range too large for values kept in key order");
  if (B == 0) B = 4ull * L + 2;  // the paper's block size
  if (B < 4ull * L + 2)
    return fail(c, LP_ERR_INVALID_ARG, "block size below 4 * ceil(log2(n + 1)) + 2");
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  if (n == 0) { *split_out = 0; return LP_OK; }
  lp::LaunchCfg cfg{sizeof(T) == 8 ? c->grid_u64 : c->grid_u32, stream, 0, nullptr};
  c->last_timed = c->timing;
  c->last_stream = stream;
  lp_status ls = ensure_var(c, lp::lowspace_implicit_scratch_bytes(cfg.grid), stream);
  if (ls != LP_OK) return ls;
  lp::TaskScratch S = c->task;
  c->last_low_tl = nullptr;
  cfg.phase_stamps = &c->last_low_tl;
  e = cudaMemsetAsync(S.status, 0, 4, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(S.bar, 0, 8, stream);
  if (c->timing && e == cudaSuccess) e = cudaEventRecord(c->ev[0], stream);
  if (e == cudaSuccess)
    e = lp::launch_lowspace_implicit<T>(keys, n, pivot, B, base_keys ? base_keys : 1,
                                        prefix_only, c->d_var, S, S.split, cfg);
  if (c->timing && e == cudaSuccess) e = cudaEventRecord(c->ev[1], stream);
  c->last_launches = cfg.launches;
  if (e != cudaSuccess) return cuda_fail(c, e, "launch");
  return read_back(c, stream, split_out);
}

}  // namespace

extern "C" {

lp_status lp_ctx_create(lp_ctx** out, int device) {
  if (!out) return LP_ERR_INVALID_ARG;
  *out = nullptr;
  lp_ctx* c = new (std::nothrow) lp_ctx();
  if (!c) return LP_ERR_OOM;
  c->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) { delete c; return LP_ERR_CUDA; }
  if ((e = lp::streaming_grid<uint64_t, false>(device, &c->grid_u64)) != cudaSuccess ||
      (e = lp::streaming_grid<uint32_t, false>(device, &c->grid_u32)) != cudaSuccess ||
      (e = lp::streaming_grid<uint64_t, true>(device, &c->grid_kv)) != cudaSuccess ||
      (e = lp::batched_prepare<uint64_t>(device, &c->grid_batch_u64)) != cudaSuccess ||
      (e = lp::batched_prepare<uint32_t>(device, &c->grid_batch_u32)) != cudaSuccess ||
      (e = lp::qs_prepare()) != cudaSuccess) {
    delete c;
    return LP_ERR_CUDA;
  }
  uint32_t gmax = c->grid_u64;
  if (c->grid_u32 > gmax) gmax = c->grid_u32;
  if (c->grid_kv > gmax) gmax = c->grid_kv;
  c->scratch_bytes = lp::task_scratch_bytes(gmax);
  e = cudaMalloc(&c->d_scratch, c->scratch_bytes);
  if (e != cudaSuccess) { delete c; return LP_ERR_OOM; }
  e = cudaMallocHost(reinterpret_cast<void**>(&c->h_pinned), 64);
  if (e != cudaSuccess) { cudaFree(c->d_scratch); delete c; return LP_ERR_OOM; }
  c->task = lp::carve_scratch(c->d_scratch, gmax);
  c->aux_bytes = c->scratch_bytes;
  *out = c;
  return LP_OK;
}

lp_status lp_ctx_destroy(lp_ctx* c) {
  if (!c) return LP_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  if (c->events_made)
    for (int i = 0; i < 3; i++) cudaEventDestroy(c->ev[i]);
  if (c->d_scratch) cudaFree(c->d_scratch);
  if (c->d_var) cudaFree(c->d_var);
  if (c->d_batch) cudaFree(c->d_batch);
  if (c->h_batch) cudaFreeHost(c->h_batch);
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  lp::hostpart_free(c);
  delete c;
  return LP_OK;
}

const char* lp_ctx_last_error(const lp_ctx* c) { return c ? c->err.c_str() : "null context"; }
uint64_t lp_ctx_aux_bytes(const lp_ctx* c) { return c ? c->aux_bytes : 0; }
uint64_t lp_ctx_last_launches(const lp_ctx* c) { return c ? c->last_launches : 0; }
uint32_t lp_ctx_grid(const lp_ctx* c) { return c ? c->grid_u64 : 0; }

lp_status lp_ctx_set_timing(lp_ctx* c, int enable) {
  if (!c) return LP_ERR_INVALID_ARG;
  if (enable) {
    lp_status s = ensure_events(c);
    if (s != LP_OK) return s;
  }
  c->timing = enable != 0;
  return LP_OK;
}

lp_status lp_ctx_set_level_cap(lp_ctx* c, uint32_t levels) {
  if (!c) return LP_ERR_INVALID_ARG;
  if (levels >= (uint32_t)lp::kMaxLevels) return fail(c, LP_ERR_INVALID_ARG, "level cap too large");
  c->level_cap = levels;
  return LP_OK;
}

lp_status lp_ctx_wait(lp_ctx* c) {
  if (!c) return LP_ERR_INVALID_ARG;
  cudaError_t e = cudaSetDevice(c->device);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->h_pinned + 7, c->task.status, 4, cudaMemcpyDeviceToHost,
                        c->last_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->last_stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "wait");
  return status_to_lp(c, (uint32_t)(c->h_pinned[7] & 0xffffffffu));
}

lp_status lp_ctx_level_stats(lp_ctx* c, uint64_t* ranges, float* ms, int* levels) {
  if (!c || !ranges || !levels) return LP_ERR_INVALID_ARG;
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  e = cudaStreamSynchronize(c->last_stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
  if (c->last_low_tl) {  // a low-space call: its phases in place of levels
    unsigned long long t[lp::kLowPhases];
    e = cudaMemcpy(t, c->last_low_tl, sizeof(t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "read phases");
    for (int L = 0; L < lp::kMaxLevels; L++) {
      for (int q = 0; q < 4; q++) ranges[4 * L + q] = 0;
      if (ms) {
        const bool have = L + 1 < lp::kLowPhases && t[L] && t[L + 1] >= t[L];
        ms[L] = have ? (float)((double)(t[L + 1] - t[L]) * 1e-6) : 0.f;
      }
    }
    *levels = lp::kMaxLevels;
    return LP_OK;
  }
  const size_t db = lp::level_desc_bytes();
  uint64_t w[lp::kMaxLevels][8];
  e = cudaMemcpy(w, c->task.desc, db * lp::kMaxLevels, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "read levels");
  uint64_t t_end = 0;
  e = cudaMemcpy(&t_end, c->task.t_end, 8, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "read end time");
  for (int L = 0; L < lp::kMaxLevels; L++) {
    ranges[4 * L + 0] = w[L][3];  // lo
    ranges[4 * L + 1] = w[L][4];  // hi
    ranges[4 * L + 2] = w[L][5];  // b
    ranges[4 * L + 3] = w[L][6];  // g
    if (ms) {
      // device timestamps: a level ends when the next one starts
      const uint64_t t0 = w[L][7];
      uint64_t t1 = (L + 1 < lp::kMaxLevels && w[L + 1][7]) ? w[L + 1][7] : t_end;
      ms[L] = (t0 && t1 > t0) ? (float)((double)(t1 - t0) * 1e-6) : 0.f;
    }
  }
  *levels = lp::kMaxLevels;
  return LP_OK;
}

lp_status lp_ctx_kernel_ms(lp_ctx* c, float* ms) {
  if (!c || !ms) return LP_ERR_INVALID_ARG;
  if (!c->last_timed) return fail(c, LP_ERR_INVALID_ARG, "the last call was not timed");
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  e = cudaEventSynchronize(c->ev[1]);
  if (e != cudaSuccess) return cuda_fail(c, e, "event synchronize");
  e = cudaEventElapsedTime(ms, c->ev[0], c->ev[1]);
  if (e != cudaSuccess) return cuda_fail(c, e, "event elapsed");
  return LP_OK;
}

lp_status lp_partition_u64(lp_ctx* c, uint64_t* keys, uint64_t n, uint64_t pivot,
                           lp_variant v, uint64_t seed, cudaStream_t s, uint64_t* split_out) {
  LP_TRACE("lp_partition_u64");
  if (!split_out) return fail(c, LP_ERR_INVALID_ARG, "null split_out");
  return partition_impl<uint64_t, false>(c, keys, nullptr, n, pivot, v, seed, s, split_out,
                                         nullptr);
}
lp_status lp_partition_u32(lp_ctx* c, uint32_t* keys, uint64_t n, uint32_t pivot,
                           lp_variant v, uint64_t seed, cudaStream_t s, uint64_t* split_out) {
  LP_TRACE("lp_partition_u32");
  if (!split_out) return fail(c, LP_ERR_INVALID_ARG, "null split_out");
  return partition_impl<uint32_t, false>(c, keys, nullptr, n, pivot, v, seed, s, split_out,
                                         nullptr);
}
lp_status lp_partition_kv_u64(lp_ctx* c, uint64_t* keys, uint64_t* vals, uint64_t n,
                              uint64_t pivot, lp_variant v, uint64_t seed, cudaStream_t s,
                              uint64_t* split_out) {
  LP_TRACE("lp_partition_kv_u64");
  if (!split_out) return fail(c, LP_ERR_INVALID_ARG, "null split_out");
  return partition_impl<uint64_t, true>(c, keys, vals, n, pivot, v, seed, s, split_out,
                                        nullptr);
}
lp_status lp_partition_u64_async(lp_ctx* c, uint64_t* keys, uint64_t n, uint64_t pivot,
                                 lp_variant v, uint64_t seed, cudaStream_t s,
                                 uint64_t* d_split) {
  LP_TRACE("lp_partition_u64_async");
  if (!d_split) return fail(c, LP_ERR_INVALID_ARG, "null d_split");
  return partition_impl<uint64_t, false>(c, keys, nullptr, n, pivot, v, seed, s, nullptr,
                                         d_split);
}
lp_status lp_partition_u32_async(lp_ctx* c, uint32_t* keys, uint64_t n, uint32_t pivot,
                                 lp_variant v, uint64_t seed, cudaStream_t s,
                                 uint64_t* d_split) {
  LP_TRACE("lp_partition_u32_async");
  if (!d_split) return fail(c, LP_ERR_INVALID_ARG, "null d_split");
  return partition_impl<uint32_t, false>(c, keys, nullptr, n, pivot, v, seed, s, nullptr,
                                         d_split);
}
lp_status lp_partition_kv_u64_async(lp_ctx* c, uint64_t* keys, uint64_t* vals, uint64_t n,
                                    uint64_t pivot, lp_variant v, uint64_t seed,
                                    cudaStream_t s, uint64_t* d_split) {
  LP_TRACE("lp_partition_kv_u64_async");
  if (!d_split) return fail(c, LP_ERR_INVALID_ARG, "null d_split");
  return partition_impl<uint64_t, true>(c, keys, vals, n, pivot, v, seed, s, nullptr, d_split);
}

lp_status lp_smoothed_step_u64(lp_ctx* c, uint64_t* keys, uint64_t n, uint64_t pivot,
                               uint64_t b, uint64_t g, uint64_t seed, uint64_t level,
                               int strided, cudaStream_t s, uint64_t* vmin, uint64_t* vmax,
                               uint64_t* count) {
  LP_TRACE("lp_smoothed_step_u64");
  return step_impl<uint64_t>(c, keys, n, pivot, b, g, seed, level, strided, s, vmin, vmax,
                             count);
}
lp_status lp_smoothed_step_u32(lp_ctx* c, uint32_t* keys, uint64_t n, uint32_t pivot,
                               uint64_t b, uint64_t g, uint64_t seed, uint64_t level,
                               int strided, cudaStream_t s, uint64_t* vmin, uint64_t* vmax,
                               uint64_t* count) {
  LP_TRACE("lp_smoothed_step_u32");
  return step_impl<uint32_t>(c, keys, n, pivot, b, g, seed, level, strided, s, vmin, vmax,
                             count);
}

lp_status lp_lowspace_partition_u64(lp_ctx* c, uint64_t* keys, uint64_t n, uint64_t pivot,
                                    uint64_t B, uint64_t base_keys, cudaStream_t s,
                                    uint64_t* split_out) {
  LP_TRACE("lp_lowspace_partition_u64");
  return lowspace_impl<uint64_t>(c, keys, n, pivot, B, base_keys, s, split_out);
}
lp_status lp_lowspace_partition_u32(lp_ctx* c, uint32_t* keys, uint64_t n, uint32_t pivot,
                                    uint64_t B, uint64_t base_keys, cudaStream_t s,
                                    uint64_t* split_out) {
  LP_TRACE("lp_lowspace_partition_u32");
  return lowspace_impl<uint32_t>(c, keys, n, pivot, B, base_keys, s, split_out);
}

lp_status lp_lowspace_implicit_partition_u64(lp_ctx* c, uint64_t* keys, uint64_t n,
                                             uint64_t pivot, uint64_t B, uint64_t base_keys,
                                             cudaStream_t s, uint64_t* split_out) {
  LP_TRACE("lp_lowspace_implicit_partition_u64");
  return implicit_impl<uint64_t>(c, keys, n, pivot, B, base_keys, 0, s, split_out);
}
lp_status lp_lowspace_implicit_partition_u32(lp_ctx* c, uint32_t* keys, uint64_t n,
                                             uint32_t pivot, uint64_t B, uint64_t base_keys,
                                             cudaStream_t s, uint64_t* split_out) {
  LP_TRACE("lp_lowspace_implicit_partition_u32");
  return implicit_impl<uint32_t>(c, keys, n, pivot, B, base_keys, 0, s, split_out);
}
lp_status lp_lowspace_implicit_prefix_u64(lp_ctx* c, uint64_t* keys, uint64_t n, uint64_t pivot,
                                          uint64_t B, cudaStream_t s, uint64_t* split_out) {
  LP_TRACE("lp_lowspace_implicit_prefix_u64");
  return implicit_impl<uint64_t>(c, keys, n, pivot, B, 0, 1, s, split_out);
}
lp_status lp_lowspace_implicit_prefix_u32(lp_ctx* c, uint32_t* keys, uint64_t n, uint32_t pivot,
                                          uint64_t B, cudaStream_t s, uint64_t* split_out) {
  LP_TRACE("lp_lowspace_implicit_prefix_u32");
  return implicit_impl<uint32_t>(c, keys, n, pivot, B, 0, 1, s, split_out);
}

lp_status lp_fill_uniform_u64(uint64_t* d, uint64_t n, uint64_t seed, cudaStream_t s) {
  if (n && !d) return LP_ERR_INVALID_ARG;
  if (!n) return LP_OK;
  return lp::launch_fill_u64(d, n, seed, s) == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}
lp_status lp_fill_uniform_u32(uint32_t* d, uint64_t n, uint64_t seed, cudaStream_t s) {
  if (n && !d) return LP_ERR_INVALID_ARG;
  if (!n) return LP_OK;
  return lp::launch_fill_u32(d, n, seed, s) == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}
lp_status lp_fill_iota_u64(uint64_t* d, uint64_t n, cudaStream_t s) {
  if (n && !d) return LP_ERR_INVALID_ARG;
  if (!n) return LP_OK;
  return lp::launch_iota_u64(d, n, s) == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}

}  // extern "C"
