/*
 * oracle.c -- plain serial CPU oracle for in-place parallel partition
 * (arXiv 2004.12532).  TEST INFRASTRUCTURE ONLY: loaded by tests/,
 * __graft_entry__.smoke() and bench.py's CPU legs, never by the product.
 *
 * Everything here is written for a reader who checks it against the paper by
 * eye: no blocking, no fusion, no reordering of the paper's steps.  Each
 * function cites the passage it follows.
 */
#include "oracle.h"
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): the state advances by the golden-ratio gamma and
 * each output is the state passed through the variant-13 finaliser.          */
static uint64_t sm64_next(uint64_t *state)
{
    uint64_t z;
    *state += 0x9E3779B97F4A7C15ull;
    z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t or_stream(uint64_t seed, uint64_t k)
{
    /* the k-th output: advance the state k times, then draw once */
    uint64_t state = seed + k * 0x9E3779B97F4A7C15ull;
    return sm64_next(&state);
}

uint64_t or_range(uint64_t r, uint64_t g)
{
    return (uint64_t)(((unsigned __int128)r * (unsigned __int128)g) >> 64);
}

/* ------------------------------------------------------------------ */
/* Sec. 2: dec(A[i]) = 1 iff A[i] is a predecessor.  Here dec(x) = [x <= pivot]. */

#define DEFINE_COUNT(NAME, T)                                              \
    uint64_t NAME(const T *a, uint64_t n, T pivot)                         \
    {                                                                      \
        uint64_t c = 0;                                                    \
        for (uint64_t i = 0; i < n; i++)                                   \
            if (a[i] <= pivot) c++;                                        \
        return c;                                                          \
    }
DEFINE_COUNT(or_count_u64, uint64_t)
DEFINE_COUNT(or_count_u32, uint32_t)

/* Serial two-pointer partition.  Invariant: a[0..i) are predecessors and
 * a[j..n) successors; each round moves i right past predecessors, j left past
 * successors, and swaps the out-of-place pair.  Ends with i == j == t.      */
#define DEFINE_PARTITION(NAME, T)                                          \
    uint64_t NAME(T *a, uint64_t n, T pivot)                               \
    {                                                                      \
        uint64_t i = 0, j = n;                                             \
        for (;;) {                                                         \
            while (i < j && a[i] <= pivot) i++;                            \
            while (i < j && a[j - 1] > pivot) j--;                         \
            if (i >= j) break;                                             \
            T tmp = a[i]; a[i] = a[j - 1]; a[j - 1] = tmp;                 \
            i++; j--;                                                      \
        }                                                                  \
        return i;                                                          \
    }
DEFINE_PARTITION(or_partition_u64, uint64_t)
DEFINE_PARTITION(or_partition_u32, uint32_t)

uint64_t or_partition_kv_u64(uint64_t *a, uint64_t *v, uint64_t n, uint64_t pivot)
{
    uint64_t i = 0, j = n;
    for (;;) {
        while (i < j && a[i] <= pivot) i++;
        while (i < j && a[j - 1] > pivot) j--;
        if (i >= j) break;
        uint64_t tk = a[i]; a[i] = a[j - 1]; a[j - 1] = tk;
        uint64_t tv = v[i]; v[i] = v[j - 1]; v[j - 1] = tv;
        i++; j--;
    }
    return i;
}

void or_partition_rows_u64(uint64_t *a, uint64_t rows, uint64_t len,
                           uint64_t pivot, uint64_t *t_out)
{
    for (uint64_t r = 0; r < rows; r++)
        t_out[r] = or_partition_u64(a + r * len, len, pivot);
}

/* ------------------------------------------------------------------ */
/* Sec. 4, "Formal Algorithm Description": X[j] uniform in the g offsets.   */
void or_draw_X(uint64_t seed, uint64_t level, uint64_t s, uint64_t g, uint64_t *X)
{
    uint64_t level_seed = or_stream(seed, level);
    for (uint64_t j = 0; j < s; j++)
        X[j] = or_range(or_stream(level_seed, j), g);
}

uint64_t or_num_chunks(uint64_t n, uint64_t b, uint64_t g)
{
    uint64_t L = (n + b - 1) / b;
    return (L + g - 1) / g;
}

/* Slots of group i, in group order: for chunk j the line
 * G_i(j) = j*g + (X[j] + i) mod g  (0-indexed form of the paper's
 * (X[j] + i mod g) + (j-1)g + 1), keys [line*b, min(line*b+b, n)).
 * Lines at or past L are the virtual padding of the footnote on
 * "n divisible by gb" and are skipped.  Returns the slot count.            */
static uint64_t group_slots(uint64_t n, uint64_t b, uint64_t g, const uint64_t *X,
                            uint64_t i, uint64_t *slot)
{
    uint64_t L = (n + b - 1) / b, s = (L + g - 1) / g, cnt = 0;
    for (uint64_t j = 0; j < s; j++) {
        uint64_t line = j * g + (X[j] + i) % g;
        if (line >= L) continue;
        uint64_t end = line * b + b < n ? line * b + b : n;
        for (uint64_t p = line * b; p < end; p++) slot[cnt++] = p;
    }
    return cnt;
}

#define DEFINE_SMOOTHED_STEP(NAME, T)                                           \
    int NAME(T *a, uint64_t n, T pivot, uint64_t b, uint64_t g, const uint64_t *X, \
             uint64_t *k, uint64_t *v, uint64_t *vmin, uint64_t *vmax)           \
    {                                                                           \
        if (b == 0 || g == 0) return -1;                                        \
        uint64_t L = (n + b - 1) / b, s = (L + g - 1) / g;                      \
        uint64_t *slot = (uint64_t *)malloc(sizeof(uint64_t) * (s * b + 1));    \
        if (!slot) return -1;                                                   \
        uint64_t lo = UINT64_MAX, hi = 0;                                       \
        for (uint64_t i = 0; i < g; i++) {                                      \
            uint64_t m = group_slots(n, b, g, X, i, slot);                      \
            /* serial partition of U_i through its slot list (same two-pointer \
               scheme as or_partition, addressed indirectly) */                 \
            uint64_t lo_p = 0, hi_p = m;                                        \
            for (;;) {                                                          \
                while (lo_p < hi_p && a[slot[lo_p]] <= pivot) lo_p++;           \
                while (lo_p < hi_p && a[slot[hi_p - 1]] > pivot) hi_p--;        \
                if (lo_p >= hi_p) break;                                        \
                T tmp = a[slot[lo_p]];                                          \
                a[slot[lo_p]] = a[slot[hi_p - 1]];                              \
                a[slot[hi_p - 1]] = tmp;                                        \
                lo_p++; hi_p--;                                                 \
            }                                                                   \
            uint64_t ki = lo_p;                                                 \
            /* v_i: index of the first successor of U_i; one past U_i's last    \
               slot when U_i holds no successor */                              \
            uint64_t vi = m == 0 ? 0 : (ki < m ? slot[ki] : slot[m - 1] + 1);   \
            if (k) k[i] = ki;                                                   \
            if (v) v[i] = vi;                                                   \
            if (m == 0) continue; /* an all-virtual group constrains nothing */ \
            if (vi < lo) lo = vi;                                               \
            if (vi > hi) hi = vi;                                               \
        }                                                                       \
        free(slot);                                                             \
        if (lo == UINT64_MAX) { lo = 0; hi = 0; }                               \
        *vmin = lo; *vmax = hi;                                                 \
        return 0;                                                               \
    }
DEFINE_SMOOTHED_STEP(or_smoothed_step_u64, uint64_t)
DEFINE_SMOOTHED_STEP(or_smoothed_step_u32, uint32_t)

/* Recursive Smoothed Striding (Sec. 4, Fig. "Smoothed Striding Algorithm"):
 * step, then recurse on A[vmin .. vmax-1]; serial once the subproblem is
 * small.                                                                    */
uint64_t or_smoothed_partition_u64(uint64_t *a, uint64_t n, uint64_t pivot,
                                   uint64_t seed, uint64_t b, uint64_t gmax,
                                   uint64_t smin, uint64_t base, uint64_t *levels)
{
    uint64_t t = or_count_u64(a, n, pivot);
    uint64_t lo = 0, hi = n, level = 0;
    if (base < 1) base = 1;
    while (hi - lo > base) {
        uint64_t m = hi - lo;
        uint64_t g = (m + b * smin - 1) / (b * smin);
        if (g > gmax) g = gmax;
        if (g < 2) g = 2;
        uint64_t s = or_num_chunks(m, b, g);
        uint64_t *X = (uint64_t *)malloc(sizeof(uint64_t) * (s ? s : 1));
        uint64_t vmin, vmax;
        or_draw_X(seed, level, s, g, X);
        or_smoothed_step_u64(a + lo, m, pivot, b, g, X, NULL, NULL, &vmin, &vmax);
        free(X);
        level++;
        if (vmax - vmin >= m) break; /* no progress: finish serially */
        hi = lo + vmax;
        lo = lo + vmin;
    }
    or_partition_u64(a + lo, hi - lo, pivot);
    if (levels) *levels = level;
    return t;
}

/* Strided Algorithm: P_i = i-th line of every chunk (X == 0), serial
 * partition of each P_i, then a serial partition of A[vmin .. vmax-1].      */
uint64_t or_strided_partition_u64(uint64_t *a, uint64_t n, uint64_t pivot,
                                  uint64_t b, uint64_t g)
{
    uint64_t t = or_count_u64(a, n, pivot);
    if (b == 0 || g == 0) return t;
    uint64_t s = or_num_chunks(n, b, g);
    uint64_t *X = (uint64_t *)calloc(s ? s : 1, sizeof(uint64_t));
    uint64_t vmin, vmax;
    or_smoothed_step_u64(a, n, pivot, b, g, X, NULL, NULL, &vmin, &vmax);
    free(X);
    or_partition_u64(a + vmin, vmax - vmin, pivot);
    return t;
}

/* ------------------------------------------------------------------ */
/* Sec. 3.  A view of the array that is either the array itself with
 * dec = [x <= pivot], or -- when predecessors are the majority -- the
 * logically reversed array A'[i] = A[n-1-i] with the roles swapped,
 * dec' = [x > pivot] (Fig. main functions, ParallelPartition).              */
typedef struct {
    uint64_t *a;
    uint64_t n;
    uint64_t pivot;
    int flip;
} view_t;

static uint64_t *at(const view_t *w, uint64_t i)
{
    return w->flip ? &w->a[w->n - 1 - i] : &w->a[i];
}
static int is_pred(const view_t *w, uint64_t x)
{
    return w->flip ? (x > w->pivot) : (x <= w->pivot);
}
static void vswap(const view_t *w, uint64_t i, uint64_t j)
{
    uint64_t *p = at(w, i), *q = at(w, j), t = *p;
    *p = *q; *q = t;
}

/* Preprocessing phase (Fig. helpers, MakeSuccessorHeavy; Lemma 3.1): for
 * i < floor(m/2) swap A[i] and A[m-1-i] when the first is a predecessor and
 * the second a successor, then repeat on the first ceil(m/2) positions.      */
static void msh_view(const view_t *w, uint64_t m)
{
    while (m > 1) {
        for (uint64_t i = 0; i < m / 2; i++)
            if (is_pred(w, *at(w, i)) && !is_pred(w, *at(w, m - 1 - i)))
                vswap(w, i, m - 1 - i);
        m = (m + 1) / 2;
    }
}

void or_make_successor_heavy_u64(uint64_t *a, uint64_t n, uint64_t pivot, int flip)
{
    view_t w = {a, n, pivot, flip};
    msh_view(&w, n);
}

/* Implicit parallel prefix sum (Fig. main functions), with the prefix values
 * stored explicitly as the paper's implementation does (Sec. 5, low-space).
 * Blocks X_1..X_{floor(n/B)}; the final block holds B..2B-1 keys.           */
static uint64_t prefix_view(const view_t *w, uint64_t B, uint64_t *v)
{
    uint64_t nb = w->n / B, acc = 0;
    for (uint64_t i = 0; i < nb; i++) {
        uint64_t start = i * B, end = (i + 1 == nb) ? w->n : start + B;
        for (uint64_t p = start; p < end; p++)
            if (is_pred(w, *at(w, p))) acc++;
        v[i] = acc;
    }
    return nb;
}

uint64_t or_block_prefix_u64(const uint64_t *a, uint64_t n, uint64_t pivot, int flip,
                             uint64_t B, uint64_t *v)
{
    view_t w = {(uint64_t *)a, n, pivot, flip};
    return prefix_view(&w, B, v);
}

/* In-place reordering (Fig. main functions, Reorder; Lemma "Reordering").
 * P = the smallest prefix of whole blocks holding at least 4/5 of the m keys;
 * partition P recursively (serially once |P| <= 5B), then swap the j-th
 * predecessor of every later block X_i into position v_{i-1} + j.          */
static void serial_partition_view(const view_t *w, uint64_t m)
{
    uint64_t i = 0, j = m;
    for (;;) {
        while (i < j && is_pred(w, *at(w, i))) i++;
        while (i < j && !is_pred(w, *at(w, j - 1))) j--;
        if (i >= j) break;
        vswap(w, i, j - 1);
        i++; j--;
    }
}

static void reorder_view(const view_t *w, uint64_t m, uint64_t B, const uint64_t *v)
{
    uint64_t nb = m / B;
    uint64_t t = (4 * m + 5 * B - 1) / (5 * B); /* least t with t*B >= 4m/5 */
    if (m <= 5 * B || t >= nb) { /* base case: small, or P would be all of A */
        serial_partition_view(w, m);
        return;
    }
    reorder_view(w, t * B, B, v);
    for (uint64_t i = t; i < nb; i++) {
        uint64_t start = i * B, end = (i + 1 == nb) ? m : start + B;
        uint64_t y = v[i - 1]; /* predecessors before X_i */
        for (uint64_t p = start; p < end; p++) {
            if (is_pred(w, *at(w, p))) {
                vswap(w, p, y);
                y++;
            }
        }
    }
}

void or_reorder_u64(uint64_t *a, uint64_t n, uint64_t pivot, int flip, uint64_t B,
                    const uint64_t *v)
{
    view_t w = {a, n, pivot, flip};
    reorder_view(&w, n, B, v);
}

uint64_t or_lowspace_partition_u64(uint64_t *a, uint64_t n, uint64_t pivot, uint64_t B)
{
    uint64_t t = or_count_u64(a, n, pivot);
    if (n == 0) return 0;
    if (B < 1) B = 1;
    /* role swap when successors are the minority */
    int flip = 2 * (n - t) < n ? 1 : 0;
    view_t w = {a, n, pivot, flip};
    msh_view(&w, n);
    uint64_t nb = n / B;
    uint64_t *v = (uint64_t *)malloc(sizeof(uint64_t) * (nb ? nb : 1));
    if (nb == 0) {
        serial_partition_view(&w, n);
    } else {
        prefix_view(&w, B, v);
        reorder_view(&w, n, B, v);
    }
    free(v);
    return t;
}

/* ------------------------------------------------------------------ */
/* Sec. 3, fully in place: the prefix values are kept in the order of the
 * keys of each block (Lemma bitstore2, which allows repeated keys), not in
 * an array.  L = ceil(log2(n + 1)) bits hold a value in [0, n]; the first
 * 4L + 2 keys of a block are read as 2L + 1 adjacent pairs.                 */
uint64_t or_bits_for(uint64_t n)
{
    uint64_t L = 0;
    while (L < 64 && (n >> L) != 0) L++; /* the bit length of n */
    return L;
}

/* Pair k of the block starting at s: positions s + 2k and s + 2k + 1. */
static void swap_pairs(const view_t *w, uint64_t s, uint64_t j, uint64_t k)
{
    vswap(w, s + 2 * j, s + 2 * k);
    vswap(w, s + 2 * j + 1, s + 2 * k + 1);
}

/* Encode v in the block at s.  On the first call the pairs are reordered
 * (keeping their relative order) so that the kind of pair that makes up at
 * least half of the 2L + 1 pairs comes first: unequal pairs (L + 1 or more)
 * give the first kind, where pair k < L holds bit k of v in its order
 * (first key > second key <=> 1); otherwise equal pairs come first, and the
 * second key of pair k, 1 <= k <= L, is overwritten with bit k - 1 of v.
 * Pair 0 tells the kinds apart: unequal for the first, equal for the second. */
static void bitstore_encode(const view_t *w, uint64_t s, uint64_t L, uint64_t v, int first)
{
    const uint64_t P = 2 * L + 1;
    if (first) {
        uint64_t unequal = 0;
        for (uint64_t k = 0; k < P; k++)
            if (*at(w, s + 2 * k) != *at(w, s + 2 * k + 1)) unequal++;
        const int want_unequal = unequal >= L + 1;
        /* stable: bubble every wanted pair down to the next free front slot */
        uint64_t front = 0;
        for (uint64_t k = 0; k < P; k++) {
            const int uneq = *at(w, s + 2 * k) != *at(w, s + 2 * k + 1);
            if (uneq == want_unequal) {
                for (uint64_t j = k; j > front; j--) swap_pairs(w, s, j - 1, j);
                front++;
            }
        }
    }
    if (*at(w, s) != *at(w, s + 1)) {
        for (uint64_t k = 0; k < L; k++) {
            uint64_t *x = at(w, s + 2 * k), *y = at(w, s + 2 * k + 1);
            const int bit = (int)((v >> k) & 1);
            const int desc = *x > *y;
            if (desc != bit) { uint64_t t = *x; *x = *y; *y = t; }
        }
    } else {
        for (uint64_t k = 1; k <= L; k++) *at(w, s + 2 * k + 1) = (v >> (k - 1)) & 1;
    }
}

/* Decode the value of the block at s; with restore, put back the keys the
 * second kind overwrote (each equals the first key of its pair).          */
static uint64_t bitstore_decode(const view_t *w, uint64_t s, uint64_t L, int restore)
{
    uint64_t v = 0;
    if (*at(w, s) != *at(w, s + 1)) {
        for (uint64_t k = 0; k < L; k++)
            if (*at(w, s + 2 * k) > *at(w, s + 2 * k + 1)) v |= 1ull << k;
    } else {
        for (uint64_t k = 1; k <= L; k++) {
            if (*at(w, s + 2 * k + 1) != 0) v |= 1ull << (k - 1);
            if (restore) *at(w, s + 2 * k + 1) = *at(w, s + 2 * k);
        }
    }
    return v;
}

void or_bitstore_encode_u64(uint64_t *x, uint64_t L, uint64_t v, int first)
{
    view_t w = {x, 4 * L + 2, 0, 0};
    bitstore_encode(&w, 0, L, v, first);
}

uint64_t or_bitstore_decode_u64(uint64_t *x, uint64_t L, int restore)
{
    view_t w = {x, 4 * L + 2, 0, 0};
    return bitstore_decode(&w, 0, L, restore);
}

/* The in-place prefix sum on values v_1..v_m kept in blocks (1-indexed, the
 * k-th value in block stride * k - 1): v_{2i} += v_{2i-1}; recurse on the
 * even-indexed values; v_{2i+1} += v_{2i}.                                  */
static void implicit_prefix_rec(const view_t *w, uint64_t B, uint64_t L, uint64_t stride,
                                uint64_t m)
{
    if (m <= 1) return;
#define BLK(k) (((k) * stride - 1) * B)
    for (uint64_t k = 2; k <= m; k += 2) {
        const uint64_t a = bitstore_decode(w, BLK(k - 1), L, 0);
        const uint64_t b = bitstore_decode(w, BLK(k), L, 0);
        bitstore_encode(w, BLK(k), L, a + b, 0);
    }
    implicit_prefix_rec(w, B, L, 2 * stride, m / 2);
    for (uint64_t k = 3; k <= m; k += 2) {
        const uint64_t a = bitstore_decode(w, BLK(k - 1), L, 0);
        const uint64_t b = bitstore_decode(w, BLK(k), L, 0);
        bitstore_encode(w, BLK(k), L, a + b, 0);
    }
#undef BLK
}

/* The prefix phase: each block first stores its own predecessor count, the
 * in-place prefix sum makes that the count in blocks 1..i, and a last pass
 * from the end moves each value one block on, so that block i ends with the
 * predecessors before it -- the value the reordering phase adds each
 * predecessor's rank to.  Returns the number of blocks floor(m/B).         */
static uint64_t implicit_prefix_view(const view_t *w, uint64_t B, uint64_t L)
{
    const uint64_t nb = w->n / B;
    for (uint64_t i = 0; i < nb; i++) {
        const uint64_t start = i * B, end = (i + 1 == nb) ? w->n : start + B;
        uint64_t c = 0;
        for (uint64_t p = start; p < end; p++)
            if (is_pred(w, *at(w, p))) c++;
        bitstore_encode(w, start, L, c, 1);
    }
    implicit_prefix_rec(w, B, L, 1, nb);
    for (uint64_t i = nb; i-- > 1;)
        bitstore_encode(w, i * B, L, bitstore_decode(w, (i - 1) * B, L, 0), 0);
    if (nb > 0) bitstore_encode(w, 0, L, 0, 0);
    return nb;
}

/* Count, role swap, MakeSuccessorHeavy and the prefix phase; the array is
 * left with every block's value encoded.  Returns t; *flip gets the role. */
uint64_t or_implicit_prefix_u64(uint64_t *a, uint64_t n, uint64_t pivot, uint64_t B, int *flip)
{
    const uint64_t t = or_count_u64(a, n, pivot);
    const int f = 2 * (n - t) < n ? 1 : 0;
    if (flip) *flip = f;
    if (n == 0) return 0;
    view_t w = {a, n, pivot, f};
    msh_view(&w, n);
    implicit_prefix_view(&w, B, or_bits_for(n));
    return t;
}

/* Reordering with the values read from the blocks (restoring overwritten
 * keys as each block is read); the base case first restores the blocks of
 * the prefix, then partitions it serially.                                */
static void implicit_reorder_view(const view_t *w, uint64_t m, uint64_t B, uint64_t L)
{
    const uint64_t nb = m / B;
    const uint64_t t = (4 * m + 5 * B - 1) / (5 * B);
    if (m <= 5 * B || t >= nb) {
        for (uint64_t i = 0; i < nb; i++) bitstore_decode(w, i * B, L, 1);
        serial_partition_view(w, m);
        return;
    }
    implicit_reorder_view(w, t * B, B, L);
    for (uint64_t i = t; i < nb; i++) {
        const uint64_t start = i * B, end = (i + 1 == nb) ? m : start + B;
        uint64_t y = bitstore_decode(w, start, L, 1); /* predecessors before X_i */
        for (uint64_t p = start; p < end; p++) {
            if (is_pred(w, *at(w, p))) {
                vswap(w, p, y);
                y++;
            }
        }
    }
}

uint64_t or_implicit_partition_u64(uint64_t *a, uint64_t n, uint64_t pivot, uint64_t B)
{
    int flip = 0;
    const uint64_t t = or_implicit_prefix_u64(a, n, pivot, B, &flip);
    if (n == 0) return 0;
    view_t w = {a, n, pivot, flip};
    implicit_reorder_view(&w, n, B, or_bits_for(n));
    return t;
}

/* ------------------------------------------------------------------ */
/* Quicksort on the partition (Sec. 5, "A Full Quicksort").  Pivot = median
 * of three seeded samples of the subarray.  When every key of the subarray is
 * <= pivot, a second partition by [x < pivot] peels off the keys equal to the
 * pivot, which are then in their final place.                               */
#define DEFINE_QUICKSORT(NAME, T, PART)                                         \
    void NAME(T *a, uint64_t n, uint64_t seed)                                  \
    {                                                                           \
        uint64_t cap = 256, top = 0;                                            \
        uint64_t *stk = (uint64_t *)malloc(sizeof(uint64_t) * 2 * cap);         \
        stk[0] = 0; stk[1] = n; top = 1;                                        \
        while (top > 0) {                                                       \
            top--;                                                              \
            uint64_t lo = stk[2 * top], hi = stk[2 * top + 1], m = hi - lo;     \
            if (m <= 16) { /* insertion sort */                                 \
                for (uint64_t i = lo + 1; i < hi; i++) {                        \
                    T x = a[i]; uint64_t j = i;                                 \
                    while (j > lo && a[j - 1] > x) { a[j] = a[j - 1]; j--; }    \
                    a[j] = x;                                                   \
                }                                                               \
                continue;                                                       \
            }                                                                   \
            uint64_t h = or_stream(seed, lo ^ (m << 32));                       \
            T s0 = a[lo + or_range(or_stream(h, 0), m)];                        \
            T s1 = a[lo + or_range(or_stream(h, 1), m)];                        \
            T s2 = a[lo + or_range(or_stream(h, 2), m)];                        \
            T p = s0 > s1 ? (s1 > s2 ? s1 : (s0 > s2 ? s2 : s0))                \
                          : (s0 > s2 ? s0 : (s1 > s2 ? s2 : s1));               \
            uint64_t t = PART(a + lo, m, p);                                    \
            uint64_t l1 = lo, h1 = lo + t, l2 = lo + t, h2 = hi;                \
            if (t == m) { /* no successor: split off keys equal to p */         \
                if (p == 0) continue; /* every key is 0: already sorted */      \
                uint64_t t2 = PART(a + lo, m, (T)(p - 1));                      \
                h1 = lo + t2; l2 = hi; h2 = hi;                                 \
            }                                                                   \
            if (top + 2 > cap) {                                                \
                cap *= 2;                                                       \
                stk = (uint64_t *)realloc(stk, sizeof(uint64_t) * 2 * cap);     \
            }                                                                   \
            if (h1 > l1 + 1) { stk[2 * top] = l1; stk[2 * top + 1] = h1; top++; } \
            if (h2 > l2 + 1) { stk[2 * top] = l2; stk[2 * top + 1] = h2; top++; } \
        }                                                                       \
        free(stk);                                                              \
    }
DEFINE_QUICKSORT(or_quicksort_u64, uint64_t, or_partition_u64)
DEFINE_QUICKSORT(or_quicksort_u32, uint32_t, or_partition_u32)
