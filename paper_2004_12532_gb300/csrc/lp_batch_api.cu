// lp_batch_api.cu -- C ABI of the batched partition (include/libpartition.h):
// the one-shot call, the graph-captured reusable batch, and the autotuner.
// All compute runs in lp_batched.cu.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "lp_batched.h"
#include "lp_ctx.h"
#include "lp_plan.h"
#include "lp_device.cuh"
#include "lp_trace.h"

struct lp_batch {
  lp_ctx* ctx = nullptr;
  uint32_t count = 0;
  uint64_t seed = 0;
  uint64_t* d_splits = nullptr;
  void* d_mem = nullptr;         // segment records, plan space, barrier and status
  lp::SegDesc* d_segs = nullptr;
  lp::BatchScratch B{};
  lp::BatchTuning tune{};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

lp::BatchTuning to_internal(const lp_batch_tuning& t) {
  lp::BatchTuning b;
  b.ctas = t.ctas;
  b.group_workers = t.group_workers;
  b.line_bytes = t.line_bytes;
  b.min_chunks = t.min_chunks;
  b.min_chunks_residual = t.min_chunks_residual;
  b.mc_slices = t.onchip_slices;
  return b;
}

lp_status check_segments(lp_ctx* c, const lp_segment_u64* segs, uint32_t count) {
  if (count && !segs) return lp_fail(c, LP_ERR_INVALID_ARG, "null segment list");
  for (uint32_t s = 0; s < count; s++) {
    if (segs[s].n && !segs[s].keys) return lp_fail(c, LP_ERR_INVALID_ARG, "null segment keys");
    if ((reinterpret_cast<uintptr_t>(segs[s].keys) & 7) != 0)
      return lp_fail(c, LP_ERR_INVALID_ARG, "segment keys not 8-byte aligned");
  }
  return LP_OK;
}

void fill_records(std::vector<lp::SegDesc>& out, const lp_segment_u64* segs, uint32_t count) {
  out.assign(count, lp::SegDesc{});
  for (uint32_t s = 0; s < count; s++) {
    out[s].keys = segs[s].keys;
    out[s].n = segs[s].n;
    out[s].pivot = segs[s].pivot;
    out[s].salt = s;  // a segment's offsets X follow from the seed and its index
  }
}

size_t records_bytes(uint32_t count) {
  return ((size_t)count * sizeof(lp::SegDesc) + 255) / 256 * 256;
}

// Grows the pinned staging buffer of the context to at least `bytes`.
lp_status ensure_staging(lp_ctx* c, size_t bytes) {
  if (bytes <= c->h_batch_bytes) return LP_OK;
  if (c->h_batch) cudaFreeHost(c->h_batch);
  c->h_batch = nullptr;
  c->h_batch_bytes = 0;
  if (cudaMallocHost(&c->h_batch, bytes) != cudaSuccess)
    return lp_fail(c, LP_ERR_OOM, "pinned staging allocation failed");
  c->h_batch_bytes = bytes;
  return LP_OK;
}

// CTAs of a batched launch: the tuned count, at most every resident CTA
uint32_t tuned_grid(const lp_ctx* c, const lp::BatchTuning& t, size_t key_bytes) {
  const uint32_t full = key_bytes == 8 ? c->grid_batch_u64 : c->grid_batch_u32;
  return t.ctas && t.ctas < full ? t.ctas : full;
}

}  // namespace

extern "C" {

lp_status lp_ctx_set_batch_tuning(lp_ctx* c, const lp_batch_tuning* t) {
  if (!c || !t) return LP_ERR_INVALID_ARG;
  if (t->line_bytes && (t->line_bytes < 128 || t->line_bytes > lp::kLineBytesMax ||
                        (t->line_bytes & 15)))
    return lp_fail(c, LP_ERR_INVALID_ARG, "line_bytes must be a multiple of 16 in 128..2048");
  c->tuning = *t;
  return LP_OK;
}

lp_status lp_partition_batched_u64(lp_ctx* c, const lp_segment_u64* segs, uint32_t count,
                                   uint64_t seed, cudaStream_t stream, uint64_t* d_splits) {
  LP_TRACE("lp_partition_batched_u64");
  if (!c) return LP_ERR_INVALID_ARG;
  c->err.clear();
  c->last_launches = 0;
  c->last_batch_traffic = nullptr;
  c->last_batch_tround = nullptr;
  if (count && !d_splits) return lp_fail(c, LP_ERR_INVALID_ARG, "null d_splits");
  lp_status st = check_segments(c, segs, count);
  if (st != LP_OK) return st;
  if (count == 0) return LP_OK;
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return lp_cuda_fail(c, e, "cudaSetDevice");
  const size_t rec = records_bytes(count), need = rec + lp::batch_scratch_bytes(count);
  // the staging buffer and the device records are reused: let earlier work
  // on this stream finish before they are rewritten
  e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return lp_cuda_fail(c, e, "stream synchronize");
  if (need > c->batch_bytes) {
    if (c->d_batch) cudaFree(c->d_batch);
    c->d_batch = nullptr;
    c->batch_bytes = 0;
    if (cudaMalloc(&c->d_batch, need) != cudaSuccess)
      return lp_fail(c, LP_ERR_OOM, "batch scratch allocation failed");
    c->batch_bytes = need;
    c->aux_bytes = c->scratch_bytes + c->var_bytes + c->batch_bytes;
  }
  if ((st = ensure_staging(c, rec)) != LP_OK) return st;
  std::vector<lp::SegDesc> recs;
  fill_records(recs, segs, count);
  memcpy(c->h_batch, recs.data(), (size_t)count * sizeof(lp::SegDesc));
  e = cudaMemcpyAsync(c->d_batch, c->h_batch, (size_t)count * sizeof(lp::SegDesc),
                      cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) return lp_cuda_fail(c, e, "upload segments");
  lp::BatchScratch B = lp::carve_batch_scratch(static_cast<unsigned char*>(c->d_batch) + rec,
                                               count, c->task.bar, c->task.status);
  const lp::BatchTuning tune = to_internal(c->tuning);
  lp::LaunchCfg cfg{tuned_grid(c, tune, 8), stream, 0, nullptr};
  c->last_timed = false;
  c->last_stream = stream;
  e = cudaMemsetAsync(c->task.status, 0, 4, stream);
  if (e != cudaSuccess) return lp_cuda_fail(c, e, "reset status");
  e = lp::launch_batched<uint64_t>(reinterpret_cast<lp::SegDesc*>(c->d_batch), count, seed,
                                   d_splits, B, tune, cfg);
  c->last_batch_traffic = B.totals + 2;
  c->last_batch_tround = B.tround;
  c->last_launches = cfg.launches;
  if (e != cudaSuccess) return lp_cuda_fail(c, e, "launch");
  return LP_OK;
}

lp_status lp_batch_create(lp_ctx* c, const lp_segment_u64* segs, uint32_t count, uint64_t seed,
                          uint64_t* d_splits, cudaStream_t stream, lp_batch** out) {
  if (!c || !out) return LP_ERR_INVALID_ARG;
  *out = nullptr;
  c->err.clear();
  if (count && !d_splits) return lp_fail(c, LP_ERR_INVALID_ARG, "null d_splits");
  lp_status st = check_segments(c, segs, count);
  if (st != LP_OK) return st;
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return lp_cuda_fail(c, e, "cudaSetDevice");
  lp_batch* b = new lp_batch();
  b->ctx = c;
  b->count = count;
  b->seed = seed;
  b->d_splits = d_splits;
  b->tune = to_internal(c->tuning);
  const size_t rec = records_bytes(count), plan = lp::batch_scratch_bytes(count);
  if (cudaMalloc(&b->d_mem, rec + plan + 256) != cudaSuccess) {
    delete b;
    return lp_fail(c, LP_ERR_OOM, "batch allocation failed");
  }
  unsigned char* base = static_cast<unsigned char*>(b->d_mem);
  b->d_segs = reinterpret_cast<lp::SegDesc*>(base);
  uint32_t* own = reinterpret_cast<uint32_t*>(base + rec + plan);  // barrier, status
  b->B = lp::carve_batch_scratch(base + rec, count, own, own + 4);
  std::vector<lp::SegDesc> recs;
  fill_records(recs, segs, count);
  if (count) {
    e = cudaMemcpy(b->d_segs, recs.data(), (size_t)count * sizeof(lp::SegDesc),
                   cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { lp_batch_destroy(b); return lp_cuda_fail(c, e, "upload segments"); }
  }
  // capture set-up, resets and the persistent launch into one graph, on a
  // stream of our own (the legacy default stream cannot be captured); the
  // graph is later launched on the caller's stream
  const uint32_t grid = tuned_grid(c, b->tune, 8);
  (void)stream;
  cudaStream_t cap = nullptr;
  e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) {
    lp::LaunchCfg cfg{grid, cap, 0, nullptr};
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t le = cudaMemsetAsync(b->B.status, 0, 4, cap);  // each launch starts clean
      if (le == cudaSuccess)
        le = lp::launch_batched<uint64_t>(b->d_segs, count, seed, d_splits, b->B, b->tune, cfg);
      e = cudaStreamEndCapture(cap, &b->graph);
      if (le != cudaSuccess) e = le;
    }
    cudaStreamDestroy(cap);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    lp_batch_destroy(b);
    return lp_cuda_fail(c, e, "graph capture of the batch");
  }
  *out = b;
  return LP_OK;
}

lp_status lp_batch_launch(lp_batch* b, cudaStream_t stream) {
  LP_TRACE("lp_batch_launch");
  if (!b) return LP_ERR_INVALID_ARG;
  if (b->count == 0) return LP_OK;
  cudaError_t e = cudaSetDevice(b->ctx->device);
  if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, stream);
  if (e != cudaSuccess) return lp_cuda_fail(b->ctx, e, "graph launch");
  b->ctx->last_launches = 2;  // kernels of the graph: set-up and the persistent kernel
  return LP_OK;
}

lp_status lp_batch_wait(lp_batch* b, cudaStream_t stream) {
  if (!b) return LP_ERR_INVALID_ARG;
  if (b->count == 0) return LP_OK;
  lp_ctx* c = b->ctx;
  cudaError_t e = cudaSetDevice(c->device);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->h_pinned + 7, b->B.status, 4, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return lp_cuda_fail(c, e, "wait");
  const uint32_t st = (uint32_t)(c->h_pinned[7] & 0xffffffffu);
  if (st & lp::kStatTimeout) return lp_fail(c, LP_ERR_TIMEOUT, lp_timeout_what(st));
  if (st) return lp_fail(c, LP_ERR_INTERNAL, "device consistency check failed");
  return LP_OK;
}

lp_status lp_batch_destroy(lp_batch* b) {
  if (!b) return LP_ERR_INVALID_ARG;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->d_mem) cudaFree(b->d_mem);
  delete b;
  return LP_OK;
}

lp_status lp_autotune_batched_u64(lp_ctx* c, const uint64_t* sizes, uint32_t count,
                                  cudaStream_t stream, lp_batch_tuning* best) {
  LP_TRACE("lp_autotune_batched_u64");
  if (!c || (count && !sizes)) return LP_ERR_INVALID_ARG;
  c->err.clear();
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return lp_cuda_fail(c, e, "cudaSetDevice");
  if (count == 0) return LP_OK;
  // a synthetic batch with these sizes, each segment 16-byte aligned
  std::vector<uint64_t> off(count);
  uint64_t total = 0;
  for (uint32_t s = 0; s < count; s++) {
    off[s] = total;
    total += (sizes[s] + 1) & ~1ull;
  }
  uint64_t* d_keys = nullptr;
  uint64_t* d_splits = nullptr;
  if (cudaMalloc(&d_keys, (total ? total : 2) * 8) != cudaSuccess ||
      cudaMalloc(&d_splits, (size_t)count * 8) != cudaSuccess) {
    if (d_keys) cudaFree(d_keys);
    return lp_fail(c, LP_ERR_OOM, "autotune buffer allocation failed");
  }
  std::vector<lp_segment_u64> segs(count);
  for (uint32_t s = 0; s < count; s++) segs[s] = {d_keys + off[s], sizes[s], 0x7fffffffffffffffull};
  const lp_batch_tuning saved = c->tuning;
  const uint32_t line_opts[] = {1024, 2048};
  const uint32_t chunk_opts[] = {16, 32, 64, 128};
  const uint32_t cta_opts[] = {0, c->grid_batch_u64 / 2};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_ms = 1e30f;
  lp_batch_tuning best_t = saved;
  lp_status st = LP_OK;
  for (uint32_t lb : line_opts)
    for (uint32_t mc : chunk_opts)
      for (uint32_t ct : cta_opts) {
        lp_batch_tuning t{ct, lb, mc, 0, 0, 0};
        c->tuning = t;
        float ms_best = 1e30f;
        for (int rep = 0; rep < 2 && st == LP_OK; rep++) {
          if (lp_fill_uniform_u64(d_keys, total, 0xA770 + rep, stream) != LP_OK) {
            st = LP_ERR_CUDA;
            break;
          }
          cudaEventRecord(e0, stream);
          st = lp_partition_batched_u64(c, segs.data(), count, 7, stream, d_splits);
          cudaEventRecord(e1, stream);
          if (cudaEventSynchronize(e1) != cudaSuccess) st = LP_ERR_CUDA;
          float ms = 0;
          cudaEventElapsedTime(&ms, e0, e1);
          if (ms < ms_best) ms_best = ms;
        }
        if (st != LP_OK) break;
        if (ms_best < best_ms) { best_ms = ms_best; best_t = t; }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d_keys);
  cudaFree(d_splits);
  c->tuning = st == LP_OK ? best_t : saved;
  if (best) *best = c->tuning;
  return st;
}

}  // extern "C"

namespace {

template <typename T>
lp_status quicksort_impl(lp_ctx* c, T* keys, uint64_t n, uint64_t seed, uint32_t samples,
                         cudaStream_t stream) {
  if (!c) return LP_ERR_INVALID_ARG;
  c->err.clear();
  c->last_launches = 0;
  if (samples != 3 && samples != 15)
    return lp_fail(c, LP_ERR_INVALID_ARG, "pivot samples must be 3 or 15");
  if (n > 0 && !keys) return lp_fail(c, LP_ERR_INVALID_ARG, "null array");
  if ((reinterpret_cast<uintptr_t>(keys) % sizeof(T)) != 0)
    return lp_fail(c, LP_ERR_INVALID_ARG, "array not aligned");
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return lp_cuda_fail(c, e, "cudaSetDevice");
  if (n < 2) return LP_OK;
  lp_status ls = ensure_var(c, lp::quicksort_scratch_bytes(n), stream);
  if (ls != LP_OK) return ls;
  e = cudaMemsetAsync(c->task.status, 0, 4, stream);
  if (e != cudaSuccess) return lp_cuda_fail(c, e, "reset status");
  const lp::BatchTuning tune = to_internal(c->tuning);
  lp::LaunchCfg cfg{tuned_grid(c, tune, sizeof(T)), stream, 0, nullptr};
  c->last_timed = false;
  c->last_stream = stream;
  c->sort_stats = lp_sort_stats{};
  if (c->timing && (ls = ensure_events(c)) != LP_OK) return ls;
  if ((ls = ensure_staging(c, lp::quicksort_staging_bytes(n))) != LP_OK) return ls;
  lp::SortStats ss{};
  e = lp::launch_quicksort<T>(keys, n, seed, samples, c->d_var, c->h_batch, tune, c->task.bar,
                              c->task.status, cfg, c->timing ? c->ev : nullptr, &ss);
  c->last_launches = cfg.launches;
  if (e != cudaSuccess) return lp_cuda_fail(c, e, "quicksort");
  c->sort_stats.levels = ss.levels;
  c->sort_stats.timed = c->timing ? 1u : 0u;
  c->sort_stats.partition_keys = ss.partition_keys;
  c->sort_stats.sort_keys = ss.sort_keys;
  c->sort_stats.partition_ms = ss.partition_ms;
  c->sort_stats.sort_ms = ss.sort_ms;
  c->sort_stats.tail_items = ss.tail_items;
  c->sort_stats.tail_ms = ss.tail_ms;
  c->sort_stats.tail_keys = ss.tail_keys;
  e = cudaMemcpyAsync(c->h_pinned, c->task.status, 4, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return lp_cuda_fail(c, e, "read status");
  const uint32_t st = (uint32_t)(c->h_pinned[0] & 0xffffffffu);
  if (st & lp::kStatTimeout) return lp_fail(c, LP_ERR_TIMEOUT, lp_timeout_what(st));
  if (st) return lp_fail(c, LP_ERR_INTERNAL, "device consistency check failed");
  return LP_OK;
}

}  // namespace

extern "C" {

lp_status lp_ctx_sort_stats(const lp_ctx* c, lp_sort_stats* out) {
  if (!c || !out) return LP_ERR_INVALID_ARG;
  *out = c->sort_stats;
  return LP_OK;
}

lp_status lp_ctx_last_batch_keys(lp_ctx* c, uint64_t* keys_out) {
  if (!c || !keys_out) return LP_ERR_INVALID_ARG;
  *keys_out = 0;
  if (!c->last_batch_traffic) return LP_OK;
  cudaError_t e = cudaSetDevice(c->device);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->h_pinned, c->last_batch_traffic, 8, cudaMemcpyDeviceToHost,
                        c->last_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->last_stream);
  if (e != cudaSuccess) return lp_cuda_fail(c, e, "read streamed keys");
  *keys_out = c->h_pinned[0];
  return LP_OK;
}

lp_status lp_batch_streamed_keys(lp_batch* b, cudaStream_t stream, uint64_t* keys_out) {
  if (!b || !keys_out) return LP_ERR_INVALID_ARG;
  *keys_out = 0;
  if (b->count == 0) return LP_OK;
  lp_ctx* c = b->ctx;
  cudaError_t e = cudaSetDevice(c->device);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->h_pinned, b->B.totals + 2, 8, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return lp_cuda_fail(c, e, "read streamed keys");
  *keys_out = c->h_pinned[0];
  return LP_OK;
}

}  // extern "C"

namespace {

lp_status read_rounds(lp_ctx* c, const unsigned long long* d_tround, cudaStream_t st,
                      lp_batch_rounds* out) {
  *out = lp_batch_rounds{};
  if (!d_tround) return LP_OK;
  static_assert(lp::kBatchRoundSlots == LP_MAX_ROUNDS, "round slots");
  unsigned long long w[LP_MAX_ROUNDS * 4];
  cudaError_t e = cudaSetDevice(c->device);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpy(w, d_tround, sizeof(w), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return lp_cuda_fail(c, e, "read round timestamps");
  for (uint32_t r = 0; r < LP_MAX_ROUNDS; r++) {
    const unsigned long long* x = w + 4 * r;
    if (!x[0]) break;
    out->rounds = r + 1;
    if (x[1] > x[0]) out->plan_ms[r] = (float)((double)(x[1] - x[0]) * 1e-6);
    if (x[2] > x[1] && x[1]) out->task_ms[r] = (float)((double)(x[2] - x[1]) * 1e-6);
    out->tasks[r] = x[3];
  }
  return LP_OK;
}

}  // namespace

extern "C" {

lp_status lp_ctx_last_batch_rounds(lp_ctx* c, lp_batch_rounds* out) {
  if (!c || !out) return LP_ERR_INVALID_ARG;
  return read_rounds(c, c->last_batch_tround, c->last_stream, out);
}

lp_status lp_batch_round_stats(lp_batch* b, cudaStream_t stream, lp_batch_rounds* out) {
  if (!b || !out) return LP_ERR_INVALID_ARG;
  return read_rounds(b->ctx, b->count ? b->B.tround : nullptr, stream, out);
}

lp_status lp_quicksort_u64(lp_ctx* c, uint64_t* keys, uint64_t n, uint64_t seed,
                           cudaStream_t stream) {
  LP_TRACE("lp_quicksort_u64");
  return quicksort_impl<uint64_t>(c, keys, n, seed, 3, stream);
}

lp_status lp_quicksort_u32(lp_ctx* c, uint32_t* keys, uint64_t n, uint64_t seed,
                           cudaStream_t stream) {
  LP_TRACE("lp_quicksort_u32");
  return quicksort_impl<uint32_t>(c, keys, n, seed, 3, stream);
}

lp_status lp_quicksort_ex_u64(lp_ctx* c, uint64_t* keys, uint64_t n, uint64_t seed,
                              uint32_t pivot_samples, cudaStream_t stream) {
  LP_TRACE("lp_quicksort_ex_u64");
  return quicksort_impl<uint64_t>(c, keys, n, seed, pivot_samples, stream);
}

lp_status lp_quicksort_ex_u32(lp_ctx* c, uint32_t* keys, uint64_t n, uint64_t seed,
                              uint32_t pivot_samples, cudaStream_t stream) {
  LP_TRACE("lp_quicksort_ex_u32");
  return quicksort_impl<uint32_t>(c, keys, n, seed, pivot_samples, stream);
}

}  // extern "C"
