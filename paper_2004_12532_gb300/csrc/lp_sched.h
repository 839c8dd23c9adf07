// lp_sched.h -- host-side pieces of the serving engine that need no GPU:
// the device-memory arena (first fit over offsets, coalescing frees) that
// enforces the HBM budget, and the FIFO admission rule.  Header-only so the
// CPU tests compile it on their own.
#pragma once
#include <stdint.h>

#include <deque>
#include <iterator>
#include <map>

namespace lp {

// Offsets into one pre-allocated device buffer of `capacity` bytes.  Every
// block is aligned to kArenaAlign bytes; alloc returns false when no free
// run is large enough (the budget is reached or fragmented).
class Arena {
 public:
  static constexpr uint64_t kArenaAlign = 256;

  explicit Arena(uint64_t capacity = 0) { reset(capacity); }

  void reset(uint64_t capacity) {
    cap_ = capacity / kArenaAlign * kArenaAlign;
    used_ = 0;
    free_.clear();
    live_.clear();
    if (cap_) free_[0] = cap_;
  }

  static uint64_t rounded(uint64_t bytes) {
    return (bytes + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
  }

  bool alloc(uint64_t bytes, uint64_t* off) {
    const uint64_t need = rounded(bytes ? bytes : 1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < need) continue;
      const uint64_t o = it->first, rest = it->second - need;
      free_.erase(it);
      if (rest) free_[o + need] = rest;
      live_[o] = need;
      used_ += need;
      *off = o;
      return true;
    }
    return false;
  }

  // Returns false for an offset that is not a live block.
  bool release(uint64_t off) {
    auto lv = live_.find(off);
    if (lv == live_.end()) return false;
    uint64_t o = off, sz = lv->second;
    live_.erase(lv);
    used_ -= sz;
    auto nx = free_.lower_bound(o);
    if (nx != free_.end() && nx->first == o + sz) {  // merge with the run after
      sz += nx->second;
      nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {  // merge with the run before
      auto pv = std::prev(nx);
      if (pv->first + pv->second == o) {
        pv->second += sz;
        return true;
      }
    }
    free_[o] = sz;
    return true;
  }

  uint64_t capacity() const { return cap_; }
  uint64_t used() const { return used_; }
  uint64_t live_blocks() const { return live_.size(); }
  uint64_t free_runs() const { return free_.size(); }
  uint64_t largest_free() const {
    uint64_t m = 0;
    for (const auto& f : free_) m = f.second > m ? f.second : m;
    return m;
  }

 private:
  uint64_t cap_ = 0, used_ = 0;
  std::map<uint64_t, uint64_t> free_;  // offset -> size
  std::map<uint64_t, uint64_t> live_;  // offset -> size
};

// FIFO admission: the head of the queue is admitted while a slot is free and
// the arena can hold its bytes; a head that does not fit blocks the ones
// behind it (no overtaking, so no request starves).  `fits` allocates and
// returns true, or returns false and changes nothing.
template <typename Fits>
uint32_t admit_fifo(std::deque<uint64_t>& queue, uint32_t free_slots, Fits&& fits,
                    uint64_t* admitted, uint32_t cap) {
  uint32_t k = 0;
  while (!queue.empty() && free_slots > 0 && k < cap) {
    if (!fits(queue.front())) break;
    admitted[k++] = queue.front();
    queue.pop_front();
    free_slots--;
  }
  return k;
}

}  // namespace lp
