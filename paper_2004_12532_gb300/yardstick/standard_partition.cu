// standard_partition.cu -- a yardstick, not the product: the Standard
// linear-space parallel partition of Sec. 2 ("The (Standard) Linear-Space
// Parallel Partition"), the paper's high-space baseline, written for the GPU.
//
//   parallel-prefix phase  S[i] = number of predecessors among A[0..i]
//                          (0-indexed, inclusive), an explicit array of n
//                          8-byte counts: per-tile counts, a scan of the tile
//                          counts, then each tile's inclusive prefix.  The
//                          decider array D is not stored: each pass applies
//                          dec(x) = [x <= pivot] to A again.
//   reordering phase       C[S[i] - 1] = A[i] for a predecessor and
//                          C[t + i - S[i]] = A[i] for a successor (the
//                          0-indexed forms of the paper's positions S[i] and
//                          t + i - S[i]), then C is copied back into A.
// Stable on both sides.  Auxiliary memory: S and C (2n 8-byte words, the
// paper's "roughly 2n eight-byte words") plus one count per tile.  bench.py
// times it beside the in-place partition; nothing in libpartition calls it.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr uint32_t kThreads = 256;
constexpr uint32_t kPer = 16;                  // keys per thread in a tile
constexpr uint32_t kTile = kThreads * kPer;    // keys per tile
constexpr uint32_t kScanThreads = 1024;

__device__ __forceinline__ uint64_t ld(const uint64_t* p) {
  return __ldg(reinterpret_cast<const unsigned long long*>(p));
}

// Exclusive scan of one value per thread over a CTA of NT threads; *total
// receives the CTA's sum.
template <uint32_t NT>
__device__ uint64_t cta_exclusive_scan(uint64_t v, uint64_t* warp_sums, uint64_t* total) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint64_t incl = v;
#pragma unroll
  for (uint32_t o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    constexpr uint32_t W = NT / 32;
    uint64_t w = lane < W ? warp_sums[lane] : 0;
    uint64_t wi = w;
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < W) warp_sums[lane] = wi - w;
    if (lane == 31) *total = wi;
  }
  __syncthreads();
  const uint64_t ex = warp_sums[warp] + incl - v;
  __syncthreads();
  return ex;
}

// Predecessor count of each tile.
__global__ void __launch_bounds__(kThreads) tile_count_kernel(const uint64_t* A, uint64_t n,
                                                              uint64_t pivot, uint64_t* tile_sum) {
  __shared__ uint64_t ws[kThreads / 32];
  __shared__ uint64_t tot;
  const uint64_t t0 = (uint64_t)blockIdx.x * kTile;
  uint64_t c = 0;
#pragma unroll
  for (uint32_t k = 0; k < kPer; k++) {
    const uint64_t i = t0 + k * kThreads + threadIdx.x;
    if (i < n) c += ld(A + i) <= pivot;
  }
  cta_exclusive_scan<kThreads>(c, ws, &tot);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

// Exclusive scan of the tile counts in place (one CTA); tile_sum[ntiles]
// receives the total t.
__global__ void __launch_bounds__(kScanThreads) tile_scan_kernel(uint64_t* tile_sum,
                                                                 uint64_t ntiles) {
  __shared__ uint64_t ws[kScanThreads / 32];
  __shared__ uint64_t tot;
  const uint64_t per = (ntiles + kScanThreads - 1) / kScanThreads;
  const uint64_t b0 = threadIdx.x * per;
  const uint64_t b1 = b0 + per < ntiles ? b0 + per : ntiles;
  uint64_t s = 0;
  for (uint64_t b = b0; b < b1; b++) s += tile_sum[b];
  uint64_t run = cta_exclusive_scan<kScanThreads>(s, ws, &tot);
  for (uint64_t b = b0; b < b1; b++) {
    const uint64_t v = tile_sum[b];
    tile_sum[b] = run;
    run += v;
  }
  if (threadIdx.x == 0) tile_sum[ntiles] = tot;
}

// S[i] for every key of each tile: the tile's offset plus the inclusive count
// within the tile (each thread owns kPer consecutive keys).
__global__ void __launch_bounds__(kThreads) tile_prefix_kernel(const uint64_t* A, uint64_t n,
                                                               uint64_t pivot,
                                                               const uint64_t* tile_off,
                                                               uint64_t* S) {
  __shared__ uint64_t ws[kThreads / 32];
  __shared__ uint64_t tot;
  const uint64_t i0 = (uint64_t)blockIdx.x * kTile + (uint64_t)threadIdx.x * kPer;
  uint32_t d = 0;  // bit k: key i0 + k is a predecessor
#pragma unroll
  for (uint32_t k = 0; k < kPer; k++)
    if (i0 + k < n && ld(A + i0 + k) <= pivot) d |= 1u << k;
  uint64_t run = tile_off[blockIdx.x] + cta_exclusive_scan<kThreads>(__popc(d), ws, &tot);
#pragma unroll
  for (uint32_t k = 0; k < kPer; k++) {
    if (i0 + k < n) {
      run += (d >> k) & 1u;
      S[i0 + k] = run;
    }
  }
}

// The reordering phase: every key to its place in C.
__global__ void reorder_kernel(const uint64_t* A, const uint64_t* S, uint64_t n, uint64_t pivot,
                               const uint64_t* total, uint64_t* C) {
  const uint64_t t = *total;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t x = ld(A + i), s = ld(S + i);
    C[x <= pivot ? s - 1 : t + i - s] = x;
  }
}

}  // namespace

extern "C" {

// Device words of scratch the Standard partition of n keys needs: S and C (n
// each) and ceil(n / 4096) + 1 tile counts.
uint64_t yd_standard_scratch_words(uint64_t n) { return 2 * n + (n + kTile - 1) / kTile + 1; }

// Partitions A[0..n) in place by [x <= pivot] through the scratch (device,
// yd_standard_scratch_words(n) words, 8-byte aligned); *d_split (device)
// receives t.  Stable: each side keeps its input order.  Stream-ordered,
// asynchronous; returns 0, or 2 on a CUDA error.
int yd_standard_partition_u64(uint64_t* A, uint64_t n, uint64_t pivot, uint64_t* scratch,
                              uint64_t* d_split, cudaStream_t stream) {
  if (n == 0) return cudaMemsetAsync(d_split, 0, 8, stream) == cudaSuccess ? 0 : 2;
  uint64_t* S = scratch;
  uint64_t* C = scratch + n;
  uint64_t* tiles = scratch + 2 * n;
  const uint64_t ntiles = (n + kTile - 1) / kTile;
  tile_count_kernel<<<(unsigned)ntiles, kThreads, 0, stream>>>(A, n, pivot, tiles);
  tile_scan_kernel<<<1, kScanThreads, 0, stream>>>(tiles, ntiles);
  tile_prefix_kernel<<<(unsigned)ntiles, kThreads, 0, stream>>>(A, n, pivot, tiles, S);
  reorder_kernel<<<152 * 16, 256, 0, stream>>>(A, S, n, pivot, tiles + ntiles, C);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(A, C, n * 8, cudaMemcpyDeviceToDevice, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_split, tiles + ntiles, 8, cudaMemcpyDeviceToDevice, stream);
  return e == cudaSuccess ? 0 : 2;
}

}  // extern "C"
