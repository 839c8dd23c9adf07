// lp_selftest.cu -- a diagnostic of the library's bounded waits: one kernel
// waits on an mbarrier phase that nothing completes and on a grid barrier
// for two CTAs in a grid of one.  Both waits must give up after the library's
// limit (about one second each) and report it, and the context must stay
// usable afterwards.  No fault, trap or endless loop is involved.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/libpartition.h"
#include "lp_device.cuh"

namespace {

__global__ void selftest_waits_kernel(uint32_t* gave_up, unsigned int* bar) {
  __shared__ __align__(8) uint64_t mb;
  __shared__ unsigned int flag;
  if (threadIdx.x == 0) {
    lp::mbar_init(&mb, 1);
    lp::fence_mbar_init();
  }
  __syncthreads();
  const bool ok1 = lp::mbar_wait_bounded(&mb, 0);  // no arrival ever comes
  if (threadIdx.x == 0) gave_up[0] = ok1 ? 0u : 1u;
  const bool ok2 = lp::grid_barrier(bar, 2u, &flag);  // the second CTA does not exist
  if (threadIdx.x == 0) gave_up[1] = ok2 ? 0u : 1u;
}

}  // namespace

extern "C" lp_status lp_selftest_bounded_waits(int device, uint32_t* mbar_gave_up,
                                              uint32_t* grid_gave_up) {
  if (!mbar_gave_up || !grid_gave_up) return LP_ERR_INVALID_ARG;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return LP_ERR_CUDA;
  void* d = nullptr;
  if (cudaMalloc(&d, 64) != cudaSuccess) return LP_ERR_OOM;
  uint32_t h[2] = {0, 0};
  e = cudaMemset(d, 0, 64);
  if (e == cudaSuccess) {
    uint32_t* words = static_cast<uint32_t*>(d);
    selftest_waits_kernel<<<1, 32>>>(words, reinterpret_cast<unsigned int*>(words + 4));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(h, d, 8, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return LP_ERR_CUDA;
  *mbar_gave_up = h[0];
  *grid_gave_up = h[1];
  return LP_OK;
}
