// cub_partition.cu -- a yardstick, not the paper's method: the out-of-place
// library partition (CUB DevicePartition::If) of the same keys by the same
// decider [x <= pivot], which needs a second array of n keys and temporary
// storage.  bench.py times it beside the in-place partition to show what the
// in-place property costs at the same bandwidth.  Built as its own library
// (libyardstick.so); nothing in libpartition calls it.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cub/device/device_partition.cuh>

namespace {

struct LessEq {
  uint64_t pivot;
  __device__ __forceinline__ bool operator()(const uint64_t& x) const { return x <= pivot; }
};

}  // namespace

extern "C" {

// Temporary storage the partition of n keys needs, in bytes.
int yd_cub_partition_temp_bytes(uint64_t n, size_t* bytes) {
  if (!bytes) return 1;
  *bytes = 0;
  cudaError_t e = cub::DevicePartition::If(nullptr, *bytes, (const uint64_t*)nullptr,
                                           (uint64_t*)nullptr, (int64_t*)nullptr, (int64_t)n,
                                           LessEq{0}, (cudaStream_t)0);
  return e == cudaSuccess ? 0 : 2;
}

// out[0..t) = keys <= pivot (input order), out[t..n) = the others (reversed);
// t is written to *d_selected (device).  Stream-ordered, asynchronous.
int yd_cub_partition_u64(const uint64_t* in, uint64_t* out, uint64_t n, uint64_t pivot,
                         int64_t* d_selected, void* temp, size_t temp_bytes,
                         cudaStream_t stream) {
  size_t tb = temp_bytes;
  cudaError_t e = cub::DevicePartition::If(temp, tb, in, out, d_selected, (int64_t)n,
                                           LessEq{pivot}, stream);
  return e == cudaSuccess ? 0 : 2;
}

}  // extern "C"
