// lp_launch.h -- internal host-side interface between the C ABI (lp_api.cu)
// and the kernel translation units.  Not part of the public API.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

namespace lp {

struct LevelDesc;

constexpr int kMaxLevels = 10;  // partial steps per partition; the last is a forced finish

// Scratch one partition task needs in device memory.
struct TaskScratch {
  LevelDesc* desc;     // kMaxLevels records
  uint32_t* status;    // device status bits
  uint64_t* split;     // where the split t is written
  uint32_t* bar;       // grid barrier: arrival count, generation
  uint32_t* counts;    // one word per CTA of the partition kernel
  unsigned long long* t_end;  // device time at the end of the last level
  uint32_t* fetch;     // per level: the next group a warp takes (kMaxLevels words)
  LevelDesc* handoff;  // [vmin, vmax): a range the recursion handed to the low-space
                       // partition (empty when it finished by itself)
};

// Bytes of TaskScratch for a partition kernel of `grid` CTAs, laid out by
// carve_scratch from a 256-byte aligned base.
size_t task_scratch_bytes(uint32_t grid);
TaskScratch carve_scratch(void* base, uint32_t grid);

struct LaunchCfg {
  uint32_t grid;       // CTAs of the streaming kernels (co-resident)
  cudaStream_t stream;
  uint64_t launches;   // incremented per kernel launch
  cudaEvent_t* events; // optional: two events around the partition kernel
  unsigned long long** phase_stamps = nullptr;  // optional: receives the low-space
                                                // kernel's phase timestamps (device)
};

// phases of the low-space kernel with a timestamp each: start, count,
// MakeSuccessorHeavy, block prefix, innermost prefix on chip, Reorder
constexpr int kLowPhases = 6;

// Keys-only (KV = false, vals == nullptr) and key+payload (KV = true, T = uint64_t).
// Full Recursive Smoothed Striding partition (strided != 0: the first step uses
// X == 0, i.e. the Strided Algorithm's partial step).
//
// Residual-shrink guard: with `handoff_var` set (lowspace_scratch_bytes(n,
// kHandoffBlock, cfg.grid) bytes), a range still open at level `level_cap`
// (1 .. kMaxLevels - 1; 0: kMaxLevels - 1), or after kShrinkTries levels
// that each left at least 7/8 of the range before them open, is handed to the
// Blocked-Prefix-Sum partition (the Hybrid of Sec. 4, Theorem 4.3) launched
// right after the recursion; it returns at once when nothing was handed over.
// Without it the last level is one group (one warp partitions what is left).
constexpr uint64_t kHandoffBlock = 4096;
constexpr int kShrinkTries = 2;
template <typename T, bool KV>
cudaError_t launch_smoothed(T* keys, uint64_t* vals, uint64_t n, T pivot, uint64_t seed,
                            int strided, const TaskScratch& S, LaunchCfg& cfg,
                            void* handoff_var = nullptr, uint32_t level_cap = 0);
// True when a partition of n keys can need the handoff (the array does not fit
// on chip at level 0).
template <typename T, bool KV>
bool smoothed_may_hand_off(uint64_t n, uint32_t grid);

// Blocked-Prefix-Sum partition (lp_lowspace.cu) of keys[lo..hi), or of the
// range [vmin, vmax) of *range_desc when it is set; the range has at most
// n_cap keys and `var` holds lowspace_scratch_bytes(n_cap, B, grid) bytes.
// split: where to write the predecessor count (may be null).
size_t lowspace_scratch_bytes(uint64_t n, uint64_t B, uint32_t grid);
template <typename T, bool KV>
cudaError_t launch_lowspace(T* keys, uint64_t* vals, uint64_t lo, uint64_t hi, uint64_t n_cap,
                            const LevelDesc* range_desc, T pivot, uint64_t B, uint64_t base_keys,
                            void* var, const TaskScratch& S, uint64_t* split, LaunchCfg& cfg);

// The same partition with the block values kept in the order of each block's
// keys (Sec. 3, Lemma bitstore2) instead of counters: keys[0..n), keys only;
// B >= 4 * lowspace_value_bits(n) + 2 and lowspace_value_bits(n) <=
// lowspace_value_bits_max().  prefix_only != 0 stops after the prefix phase,
// leaving every block's value encoded.  `var` holds
// lowspace_implicit_scratch_bytes(grid) bytes.
size_t lowspace_implicit_scratch_bytes(uint32_t grid);
uint32_t lowspace_value_bits(uint64_t n);
uint32_t lowspace_value_bits_max();
template <typename T>
cudaError_t launch_lowspace_implicit(T* keys, uint64_t n, T pivot, uint64_t B,
                                     uint64_t base_keys, int prefix_only, void* var,
                                     const TaskScratch& S, uint64_t* split, LaunchCfg& cfg);

// Smoothed Striding level 0 only (the Strided Algorithm's partial step when
// strided != 0), leaving [vmin, vmax) in S.desc[0] for a cleanup; then
// finalize_smoothed places the unaligned head and tail and writes the split.
template <typename T, bool KV>
cudaError_t launch_first_level(T* keys, uint64_t* vals, uint64_t n, T pivot, uint64_t seed,
                               int strided, const TaskScratch& S, LaunchCfg& cfg, uint64_t* h,
                               uint64_t* body_end);
template <typename T, bool KV>
cudaError_t launch_finalize(T* keys, uint64_t* vals, uint64_t n, uint64_t h, uint64_t body_end,
                            T pivot, const TaskScratch& S, LaunchCfg& cfg);

// One Partial Partition Step with explicit parameters over keys[0..n).
template <typename T>
cudaError_t launch_step(T* keys, uint64_t n, T pivot, uint64_t b, uint64_t g, uint64_t seed,
                        uint64_t level, int strided, const TaskScratch& S, LaunchCfg& cfg);

// Occupancy-derived grid for the streaming kernels.
template <typename T, bool KV>
cudaError_t streaming_grid(int device, uint32_t* grid);

uint64_t small_limit(uint32_t key_bytes, bool kv);

cudaError_t launch_fill_u64(uint64_t* d, uint64_t n, uint64_t seed, cudaStream_t s);
cudaError_t launch_fill_u32(uint32_t* d, uint64_t n, uint64_t seed, cudaStream_t s);
cudaError_t launch_iota_u64(uint64_t* d, uint64_t n, cudaStream_t s);

// Size of one LevelDesc (the struct is opaque to lp_api.cu).
size_t level_desc_bytes();

}  // namespace lp
