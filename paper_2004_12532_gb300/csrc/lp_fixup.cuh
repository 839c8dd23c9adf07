// lp_fixup.cuh -- the head and tail of a range whose 16-byte aligned body the
// partition kernels partitioned: shared by the batched engine and the
// quicksort's on-chip finishing kernel.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lp {

template <typename T>
__device__ __forceinline__ T ldk(const T* p) {
  if constexpr (sizeof(T) == 8) return (T)__ldcg(reinterpret_cast<const unsigned long long*>(p));
  else return (T)__ldcg(reinterpret_cast<const unsigned int*>(p));
}

// Places the (< 16-byte) unaligned head [0, h) and tail [be, n) of a segment
// whose aligned body [h, be) is partitioned with body_count predecessors;
// returns the split.  One thread.
template <typename T>
__device__ uint64_t seg_fixup(T* keys, uint64_t n, uint64_t h, uint64_t be, uint64_t body_count,
                              T pivot) {
  const uint64_t m = h + body_count;
  uint64_t hp = 0, tp = 0;
  for (uint64_t p = 0; p < h; p++) hp += ldk(&keys[p]) <= pivot;
  for (uint64_t p = be; p < n; p++) tp += ldk(&keys[p]) <= pivot;
  const uint64_t t = body_count + hp + tp;
  uint64_t bad_s[16], bad_p[16];
  int ns = 0, np = 0;
  auto visit = [&](uint64_t p) {
    const bool pr = ldk(&keys[p]) <= pivot;
    if (p < t && !pr && ns < 16) bad_s[ns++] = p;
    if (p >= t && pr && np < 16) bad_p[np++] = p;
  };
  for (uint64_t p = 0; p < h; p++) visit(p);
  uint64_t r0 = m < t ? m : t, r1 = m < t ? t : m;
  if (r0 < h) r0 = h;
  if (r1 > be) r1 = be;
  for (uint64_t p = r0; p < r1; p++) visit(p);
  for (uint64_t p = be; p < n; p++) visit(p);
  const int q = ns < np ? ns : np;
  for (int j = 0; j < q; j++) {
    const T x = ldk(&keys[bad_s[j]]);
    keys[bad_s[j]] = ldk(&keys[bad_p[j]]);
    keys[bad_p[j]] = x;
  }
  return t;
}

}  // namespace lp
