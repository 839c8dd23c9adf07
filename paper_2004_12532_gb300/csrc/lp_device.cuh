// lp_device.cuh -- sm_103a device helpers written as inline PTX: mbarriers,
// 1-D bulk asynchronous copies (the non-tensor TMA path) between global and
// shared memory, proxy fences, and a bounded wait.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

namespace lp {

// Status bits a kernel may raise in its status word (host maps them to
// lp_status codes).
enum : uint32_t {
  kStatTimeout = 1u,     // a bounded wait gave up
  kStatRing = 2u,        // ring capacity check failed (never expected)
  kStatUnfinished = 4u,  // a range was still open after the last level
  kStatBadArg = 8u,
};
// Where a bounded wait gave up: raised with kStatTimeout, one bit per kind of
// wait, so that the host can say which one.
enum : uint32_t {
  kSitePartition = 1u << 16,  // a grid barrier of the single partition
  kSiteLowspace = 1u << 17,   // a grid barrier of the low-space partition
  kSiteRounds = 1u << 18,     // a grid barrier of the batched engine's rounds
  kSiteSortLoop = 1u << 19,   // a grid barrier of the quicksort's level loop
  kSiteLine = 1u << 20,       // a warp's wait for a line's bulk copy
  kSiteBulk = 1u << 21,       // a CTA's wait for a range's bulk copy
};

// Wall-clock limit of any single wait, in ns (about one second).
constexpr uint64_t kWaitLimitNs = 1000000000ull;

// Limit of a grid barrier that follows work on `bytes` bytes which some CTA may
// stream alone (a one-group step is one warp's partition of a whole range):
// the fixed limit plus 2 ns per byte, i.e. a floor of 0.5 GB/s for that CTA,
// so that slow but correct work never gives up.
__host__ __device__ __forceinline__ uint64_t wait_limit_for_bytes(uint64_t bytes) {
  return kWaitLimitNs + 2ull * bytes;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

// Ends an mbarrier's life so its shared memory may be reused for data.
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's generic-proxy shared-memory writes before later
// async-proxy (bulk copy) reads of the same bytes.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Orders this thread's generic-proxy global-memory accesses before later
// async-proxy (bulk copy) accesses of the same bytes.
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for completion of phase `parity` of `bar`, for at most kWaitLimitNs.
// Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  uint64_t t0 = global_timer_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_timer_ns() - t0 > kWaitLimitNs) return false;
  }
}

// Global -> shared bulk copy completing on `bar` (bytes: multiple of 16, both
// addresses 16-byte aligned).
__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst_smem)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Shared -> global bulk copy tracked by the issuing thread's bulk groups.
__device__ __forceinline__ void bulk_store(void* dst, const void* src_smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_addr(src_smem)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Wait until at most N committed bulk groups of this thread still read smem.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

// Wait until at most N committed bulk groups of this thread are incomplete.
template <int N>
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).  bar[0]
// counts arrivals, bar[1] is the generation; both start at zero.  The last
// CTA to arrive resets the count and advances the generation; the others wait
// for the generation to change, for at most limit_ns.  Returns false (in
// every thread of the CTA) if this CTA gave up waiting.  Proxy fences on both
// sides order the plain stores before the barrier with the bulk copies
// (async proxy) after it, in every CTA.
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, unsigned int nblocks,
                                             unsigned int* flag_smem,
                                             uint64_t limit_ns = kWaitLimitNs) {
  fence_proxy_async_global();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int ok = 1u;
    volatile unsigned int* gen = bar + 1;
    const unsigned int g0 = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == nblocks - 1u) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const uint64_t t0 = global_timer_ns();
      while (*gen == g0) {
        if (global_timer_ns() - t0 > limit_ns) { ok = 0u; break; }
        __nanosleep(64);
      }
    }
    __threadfence();
    *flag_smem = ok;
  }
  __syncthreads();
  fence_proxy_async_global();
  return *flag_smem != 0u;
}

// Launches a kernel whose CTAs wait on one another (grid_barrier): the
// cooperative launch attribute makes the runtime guarantee that all `grid`
// CTAs are resident at once (or fail the launch), and this form of launch can
// be captured into a CUDA graph.
template <typename... P, typename... A>
inline cudaError_t launch_cooperative(void (*kernel)(P...), uint32_t grid, uint32_t threads,
                                      size_t smem, cudaStream_t stream, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace lp
