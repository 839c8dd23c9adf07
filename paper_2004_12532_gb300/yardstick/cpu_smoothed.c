/* cpu_smoothed.c -- a yardstick, not the product: the Smoothed Striding
 * partition (Sec. 4) on the host's cores with OpenMP, the paper's own setting,
 * timed by bench.py beside the serial CPU baseline and the GPU.  Built as its
 * own library (libcpuyard.so); nothing in libpartition calls it.
 *
 * One Partial Partition Step over the first s*g*b keys (s chunks of g lines of
 * b keys; group i takes line j*g + (X[j] + i) mod g of chunk j; the groups are
 * partitioned serially and in parallel, each by a two-pointer scan over its
 * slots; v_i = the position of slot k_i of group i), the tail of fewer than
 * g*b keys partitioned serially; the open range [min v_i, max v_i) is
 * partitioned the same way, recursively, and serially once it is small; the
 * tail's predecessors are finally swapped in after the open range's. */
#include <stdint.h>
#include <stdlib.h>

#include <omp.h>

static uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* serial two-pointer partition of a[0..n) by [x <= pivot]; returns the count */
static uint64_t serial_partition(uint64_t* a, uint64_t n, uint64_t pivot) {
  uint64_t lo = 0, hi = n;
  for (;;) {
    while (lo < hi && a[lo] <= pivot) lo++;
    while (lo < hi && a[hi - 1] > pivot) hi--;
    if (lo >= hi) return lo;
    const uint64_t t = a[lo];
    a[lo] = a[hi - 1];
    a[hi - 1] = t;
    lo++;
    hi--;
  }
}

typedef struct {
  uint64_t* a;
  uint64_t b, g, s;
  const uint32_t* X;
} step_t;

static inline uint64_t slot_pos(const step_t* S, uint64_t i, uint64_t k) {
  const uint64_t j = k / S->b, off = k % S->b;
  uint64_t x = S->X[j] + i;
  if (x >= S->g) x -= S->g;
  return (j * S->g + x) * S->b + off;
}

/* partitions group i in slot order; returns k_i */
static uint64_t group_partition(const step_t* S, uint64_t i, uint64_t pivot) {
  uint64_t lo = 0, hi = S->s * S->b;
  for (;;) {
    while (lo < hi && S->a[slot_pos(S, i, lo)] <= pivot) lo++;
    while (lo < hi && S->a[slot_pos(S, i, hi - 1)] > pivot) hi--;
    if (lo >= hi) return lo;
    const uint64_t p = slot_pos(S, i, lo), q = slot_pos(S, i, hi - 1);
    const uint64_t t = S->a[p];
    S->a[p] = S->a[q];
    S->a[q] = t;
    lo++;
    hi--;
  }
}

static uint64_t smoothed(uint64_t* a, uint64_t n, uint64_t pivot, int threads, uint64_t seed,
                         uint64_t level) {
  const uint64_t b = 512, min_chunks = 64;
  uint64_t g = n / (b * min_chunks);
  if (g > (uint64_t)threads * 16) g = (uint64_t)threads * 16;
  if (g < 2 || n < (1u << 16)) return serial_partition(a, n, pivot);
  const uint64_t s = n / (g * b), region = s * g * b;
  uint32_t* X = (uint32_t*)malloc(s * sizeof(uint32_t));
  if (!X) return serial_partition(a, n, pivot);
  const uint64_t sig = sm_mix(seed + (level + 1) * 0x9E3779B97F4A7C15ull);
  for (uint64_t j = 0; j < s; j++)
    X[j] = (uint32_t)(((unsigned __int128)sm_mix(sig + (j + 1) * 0x9E3779B97F4A7C15ull) * g) >> 64);
  step_t S = {a, b, g, s, X};
  uint64_t vmin = region, vmax = 0;
#pragma omp parallel for num_threads(threads) schedule(dynamic, 1) \
    reduction(min : vmin) reduction(max : vmax)
  for (int64_t i = 0; i < (int64_t)g; i++) {
    const uint64_t k = group_partition(&S, (uint64_t)i, pivot);
    const uint64_t v = k < s * b ? slot_pos(&S, (uint64_t)i, k)
                                 : slot_pos(&S, (uint64_t)i, s * b - 1) + 1;
    if (v < vmin) vmin = v;
    if (v > vmax) vmax = v;
  }
  free(X);
  /* [0, vmin) predecessors, [vmax, region) successors, [vmin, vmax) open */
  const uint64_t tp = serial_partition(a + region, n - region, pivot);
  const uint64_t cm = vmax > vmin ? smoothed(a + vmin, vmax - vmin, pivot, threads, seed,
                                             level + 1)
                                  : 0;
  /* [first_succ, region) successors, then the tail's tp predecessors: swap
     the first k successors with the last k of those predecessors */
  const uint64_t first_succ = vmin + cm, ls = region - first_succ;
  const uint64_t k = ls < tp ? ls : tp;
  for (uint64_t q = 0; q < k; q++) {
    const uint64_t p = first_succ + q, r = region + tp - k + q;
    const uint64_t t = a[p];
    a[p] = a[r];
    a[r] = t;
  }
  return first_succ + tp;
}

/* Partitions a[0..n) by [x <= pivot] with `threads` threads; returns the count. */
uint64_t cy_smoothed_partition_u64(uint64_t* a, uint64_t n, uint64_t pivot, int threads,
                                   uint64_t seed) {
  return smoothed(a, n, pivot, threads < 1 ? 1 : threads, seed, 0);
}
