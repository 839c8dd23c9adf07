// lp_noalloc.cu -- lp_partition_u64_noalloc: the Smoothed Striding / Strided
// partition of uint64 keys without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// partition: code running inside another allocator's callback, latency-bound
// loops where the implicit device synchronisation of cudaMalloc is not
// acceptable, and processes whose device memory is entirely reserved by a
// framework's caching pool.  They cannot create an lp_ctx (which allocates its
// scratch), so this entry point keeps the scratch the partition needs -- the
// per-level descriptors, a status word, the grid barrier and one count per CTA
// of the launch, about 2 KB on a 152-SM GPU -- in a file-scope __device__
// array instead.  It launches the Smoothed Striding kernels of
// lp_partition_u64_async and calls no allocating routine.  Without counters
// for the low-space partition it cannot hand a range over: a range still open
// at the last level is finished by one group, and LP_STRIDED is the Strided
// first step followed by the Smoothed Striding recursion.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/libpartition.h"
#include "lp_launch.h"

namespace {

constexpr size_t kScratchBytes = LP_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// Shared by every call on a device; holds the last call's descriptors.
__device__ __align__(256) unsigned char noalloc_scratch[kScratchBytes];

struct DeviceSetup {
  bool done = false;
  void* scratch = nullptr;  // device address of noalloc_scratch on this device
  uint32_t grid = 0;
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;


// Once per device, with that device current: resolve the array's device
// address and the launch grid.  No allocation.
lp_status setup_device(int dev, DeviceSetup** out) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  DeviceSetup& d = g_setup[dev];
  if (!d.done) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, noalloc_scratch) != cudaSuccess) return LP_ERR_CUDA;
    uint32_t grid = 0;
    if (lp::streaming_grid<uint64_t, false>(dev, &grid) != cudaSuccess) return LP_ERR_CUDA;
    d.scratch = p;
    d.grid = grid;
    d.done = true;
  }
  *out = &d;
  return LP_OK;
}

}  // namespace

extern "C" lp_status lp_partition_u64_noalloc(uint64_t* keys, uint64_t n, uint64_t pivot,
                                              lp_variant variant, uint64_t seed,
                                              cudaStream_t stream, uint64_t* d_split) {
  if (!d_split) return LP_ERR_INVALID_ARG;
  if (n > 0 && !keys) return LP_ERR_INVALID_ARG;
  if (variant != LP_SMOOTHED && variant != LP_STRIDED) return LP_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(keys) & 7) != 0) return LP_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LP_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return LP_ERR_INVALID_ARG;
  if (n == 0) return cudaMemsetAsync(d_split, 0, 8, stream) == cudaSuccess ? LP_OK : LP_ERR_CUDA;
  DeviceSetup* d = nullptr;
  const lp_status st = setup_device(dev, &d);
  if (st != LP_OK) return st;
  // the scratch grows with the launch grid (one word per CTA): refuse a
  // device whose grid needs more than the array holds
  if (lp::task_scratch_bytes(d->grid) > kScratchBytes) return LP_ERR_INVALID_ARG;
  lp::TaskScratch S = lp::carve_scratch(d->scratch, d->grid);
  S.split = d_split;
  lp::LaunchCfg cfg{d->grid, stream, 0, nullptr};
  const cudaError_t e = lp::launch_smoothed<uint64_t, false>(
      keys, nullptr, n, pivot, seed, variant == LP_STRIDED ? 1 : 0, S, cfg);
  return e == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}
