// lp_hostpart.cu -- lp_partition_host_u64 / _u32: the partition of an array
// held in host memory.  Chunks go to the device on one stream; each is
// partitioned there in place by the Smoothed Striding partition (one
// cooperative launch, lp_kernels.cu) on a second stream; a third stream copies
// the predecessors and successors of the partitioned chunks back to their
// final places in the host array as the plan (lp_hostpart.h) allows, so the
// copies in both directions overlap.  Host code only; every key is moved by
// the copy engines and partitioned by the library's kernels.
#include <cuda_runtime.h>
#include <stdint.h>

#include <new>
#include <vector>

#include "../../include/libpartition.h"
#include "lp_ctx.h"
#include "lp_device.cuh"
#include "lp_hostpart.h"
#include "lp_launch.h"
#include "lp_trace.h"

namespace lp {

namespace {

constexpr uint32_t kHostLag = 2;        // an upload's side uses counts this many uploads old
constexpr uint32_t kHostAhead = 4;      // uploads in flight ahead of the partitions, at most
constexpr uint64_t kHostChunkMin = 1ull << 22;  // keys per chunk, at least
constexpr uint32_t kHostChunks = 32;    // chunks per array, about

uint64_t host_chunk_keys(uint64_t n) {
  uint64_t c = (n + kHostChunks - 1) / kHostChunks;
  c = (c + 4095) / 4096 * 4096;
  return c < kHostChunkMin ? kHostChunkMin : c;
}

}  // namespace

struct HostPart {
  void* d_buf = nullptr;   // the device copy of the array
  size_t d_bytes = 0;
  bool streams = false;
  cudaStream_t s_up = nullptr, s_comp = nullptr, s_down = nullptr;
  cudaEvent_t ev_start = nullptr, ev_end = nullptr;
  std::vector<cudaEvent_t> ev_up, ev_part;  // per upload
  uint64_t* h_slots = nullptr;              // pinned: split and status per upload
  size_t n_slots = 0;
};

void hostpart_free(lp_ctx* c) {
  HostPart* H = static_cast<HostPart*>(c->hostpart);
  if (!H) return;
  if (H->d_buf) cudaFree(H->d_buf);
  if (H->h_slots) cudaFreeHost(H->h_slots);
  for (cudaEvent_t e : H->ev_up) cudaEventDestroy(e);
  for (cudaEvent_t e : H->ev_part) cudaEventDestroy(e);
  if (H->streams) {
    cudaEventDestroy(H->ev_start);
    cudaEventDestroy(H->ev_end);
    cudaStreamDestroy(H->s_up);
    cudaStreamDestroy(H->s_comp);
    cudaStreamDestroy(H->s_down);
  }
  delete H;
  c->hostpart = nullptr;
}

namespace {

lp_status host_setup(lp_ctx* c, HostPart& H, size_t bytes, uint32_t K, cudaStream_t stream) {
  cudaError_t e;
  if (!H.streams) {
    if ((e = cudaStreamCreateWithFlags(&H.s_up, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&H.s_comp, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&H.s_down, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&H.ev_start, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&H.ev_end, cudaEventDisableTiming)) != cudaSuccess)
      return lp_cuda_fail(c, e, "streams");
    H.streams = true;
  }
  if (H.d_bytes < bytes) {
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return lp_cuda_fail(c, e, "sync");
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return lp_cuda_fail(c, e, "sync");
    if (H.d_buf) cudaFree(H.d_buf);
    H.d_buf = nullptr;
    H.d_bytes = 0;
    if (cudaMalloc(&H.d_buf, bytes) != cudaSuccess) {
      cudaGetLastError();
      return lp_fail(c, LP_ERR_OOM, "device copy of the host array");
    }
    H.d_bytes = bytes;
  }
  while (H.ev_up.size() < K) {
    cudaEvent_t a, b;
    if ((e = cudaEventCreateWithFlags(&a, cudaEventDisableTiming)) != cudaSuccess)
      return lp_cuda_fail(c, e, "events");
    if ((e = cudaEventCreateWithFlags(&b, cudaEventDisableTiming)) != cudaSuccess) {
      cudaEventDestroy(a);
      return lp_cuda_fail(c, e, "events");
    }
    H.ev_up.push_back(a);
    H.ev_part.push_back(b);
  }
  if (H.n_slots < 2 * (size_t)K) {
    if (H.h_slots) cudaFreeHost(H.h_slots);
    H.h_slots = nullptr;
    H.n_slots = 0;
    if (cudaHostAlloc(reinterpret_cast<void**>(&H.h_slots), 16 * (size_t)K, cudaHostAllocDefault) !=
        cudaSuccess) {
      cudaGetLastError();
      return lp_fail(c, LP_ERR_OOM, "pinned read-back slots");
    }
    H.n_slots = 2 * (size_t)K;
  }
  return LP_OK;
}

template <typename T>
lp_status host_partition(lp_ctx* c, T* host, uint64_t n, T pivot, uint64_t seed,
                         cudaStream_t stream, uint64_t* split_out) {
  if (!c) return LP_ERR_INVALID_ARG;
  c->err.clear();
  c->last_launches = 0;
  c->last_timed = false;
  c->last_low_tl = nullptr;
  if (!split_out) return lp_fail(c, LP_ERR_INVALID_ARG, "null split_out");
  if (n > 0 && !host) return lp_fail(c, LP_ERR_INVALID_ARG, "null array");
  if (reinterpret_cast<uintptr_t>(host) % sizeof(T) != 0)
    return lp_fail(c, LP_ERR_INVALID_ARG, "array not naturally aligned");
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return lp_cuda_fail(c, e, "cudaSetDevice");
  if (n == 0) {
    *split_out = 0;
    return LP_OK;
  }
  if (!c->hostpart) {
    c->hostpart = new (std::nothrow) HostPart();
    if (!c->hostpart) return lp_fail(c, LP_ERR_OOM, "host partition state");
  }
  HostPart& H = *static_cast<HostPart*>(c->hostpart);
  HostChunkPlan plan;
  plan.init(n, host_chunk_keys(n), kHostLag);
  const uint32_t K = plan.chunks();
  lp_status ls = host_setup(c, H, (size_t)n * sizeof(T), K, stream);
  if (ls != LP_OK) return ls;
  c->last_stream = stream;
  // after the caller's earlier work on `stream`
  if ((e = cudaEventRecord(H.ev_start, stream)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(H.s_up, H.ev_start, 0)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(H.s_comp, H.ev_start, 0)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(H.s_down, H.ev_start, 0)) != cudaSuccess)
    return lp_cuda_fail(c, e, "order after the caller's stream");
  // an error after copies were queued: let them finish before returning, so
  // nothing writes the caller's host array after the call
  auto bail = [&](lp_status st) {
    cudaStreamSynchronize(H.s_up);
    cudaStreamSynchronize(H.s_comp);
    cudaStreamSynchronize(H.s_down);
    return st;
  };
  T* dev = static_cast<T*>(H.d_buf);
  TaskScratch S = c->task;
  LaunchCfg cfg{sizeof(T) == 8 ? c->grid_u64 : c->grid_u32, H.s_comp, 0, nullptr};
  std::vector<HostPiece> pieces;
  uint32_t status = 0;
  while (!plan.finished()) {
    while (plan.uploads() < K && plan.processed() >= plan.needed_for_next() &&
           plan.uploads() - plan.processed() < kHostAhead) {
      const uint32_t j = plan.uploads();
      const uint32_t k = plan.next_upload();
      const uint64_t b = plan.chunk_begin(k), len = plan.chunk_len(k);
      H.h_slots[2 * j] = 0;
      H.h_slots[2 * j + 1] = 0;
      if ((e = cudaMemcpyAsync(dev + b, host + b, len * sizeof(T), cudaMemcpyHostToDevice,
                               H.s_up)) != cudaSuccess ||
          (e = cudaEventRecord(H.ev_up[j], H.s_up)) != cudaSuccess ||
          (e = cudaStreamWaitEvent(H.s_comp, H.ev_up[j], 0)) != cudaSuccess)
        return bail(lp_cuda_fail(c, e, "upload"));
      if ((e = launch_smoothed<T, false>(dev + b, nullptr, len, pivot, seed + k, 0, S, cfg)) !=
          cudaSuccess)
        return bail(lp_cuda_fail(c, e, "partition of a chunk"));
      if ((e = cudaMemcpyAsync(H.h_slots + 2 * j, S.split, 8, cudaMemcpyDeviceToHost,
                               H.s_comp)) != cudaSuccess ||
          (e = cudaMemcpyAsync(H.h_slots + 2 * j + 1, S.status, 4, cudaMemcpyDeviceToHost,
                               H.s_comp)) != cudaSuccess ||
          (e = cudaEventRecord(H.ev_part[j], H.s_comp)) != cudaSuccess)
        return bail(lp_cuda_fail(c, e, "read a chunk's split"));
    }
    const uint32_t j = plan.processed();
    if (j >= plan.uploads())
      return bail(lp_fail(c, LP_ERR_INTERNAL, "host partition plan stalled"));
    if ((e = cudaEventSynchronize(H.ev_part[j])) != cudaSuccess)
      return bail(lp_cuda_fail(c, e, "partition of a chunk"));
    // a chunk whose partition failed on the device, or whose split cannot be
    // one, plans no copy back: stop before the caller's array is written from it
    status |= (uint32_t)(H.h_slots[2 * j + 1] & 0xffffffffu);
    if (status & kStatTimeout) return bail(lp_fail(c, LP_ERR_TIMEOUT, lp_timeout_what(status)));
    if (status) return bail(lp_fail(c, LP_ERR_INTERNAL, "device consistency check failed"));
    if (!plan.partitioned(H.h_slots[2 * j]))
      return bail(lp_fail(c, LP_ERR_INTERNAL, "a chunk's split exceeds its length"));
    pieces.clear();
    plan.take_pieces(pieces);
    if (!pieces.empty() && (e = cudaStreamWaitEvent(H.s_down, H.ev_part[j], 0)) != cudaSuccess)
      return bail(lp_cuda_fail(c, e, "order the copies back"));
    for (const HostPiece& p : pieces)
      if ((e = cudaMemcpyAsync(host + p.host, dev + p.dev, p.len * sizeof(T),
                               cudaMemcpyDeviceToHost, H.s_down)) != cudaSuccess)
        return bail(lp_cuda_fail(c, e, "copy back"));
  }
  if ((e = cudaEventRecord(H.ev_end, H.s_down)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(stream, H.ev_end, 0)) != cudaSuccess ||
      (e = cudaEventSynchronize(H.ev_end)) != cudaSuccess)
    return bail(lp_cuda_fail(c, e, "finish the copies back"));
  c->last_launches = cfg.launches;
  *split_out = plan.split();
  if (status & kStatTimeout) return lp_fail(c, LP_ERR_TIMEOUT, lp_timeout_what(status));
  if (status) return lp_fail(c, LP_ERR_INTERNAL, "device consistency check failed");
  return LP_OK;
}

}  // namespace

}  // namespace lp

extern "C" {

lp_status lp_partition_host_u64(lp_ctx* c, uint64_t* keys, uint64_t n, uint64_t pivot,
                                uint64_t seed, cudaStream_t stream, uint64_t* split_out) {
  LP_TRACE("lp_partition_host_u64");
  return lp::host_partition<uint64_t>(c, keys, n, pivot, seed, stream, split_out);
}

lp_status lp_partition_host_u32(lp_ctx* c, uint32_t* keys, uint64_t n, uint32_t pivot,
                                uint64_t seed, cudaStream_t stream, uint64_t* split_out) {
  LP_TRACE("lp_partition_host_u32");
  return lp::host_partition<uint32_t>(c, keys, n, pivot, seed, stream, split_out);
}

}  // extern "C"
