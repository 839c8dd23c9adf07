// lp_hostpart.h -- the plan of a partition of an array in host memory (no
// counterpart in the paper: it feeds the device partition of Sec. 4 from the
// host).  Pure host code, shared by the library (lp_hostpart.cu) and its CPU
// test (tests/csrc/hostpart_test.cpp).
//
// The array of n keys is cut into K chunks of C keys (the last one shorter).
// Chunks go to the device one at a time, taken from the front or the back of
// the array; each is partitioned on the device in place, and then its p
// predecessors belong at the next p free positions from the front of the
// host array and its s successors at the next s free positions from the back.
// A host position may be written only once its own chunk has reached the
// device (its input is consumed): the plan hands out the device-to-host
// copies as they become legal, in pieces.  The side of the j-th upload is the
// side with more output waiting, computed from the counts of the first
// j + 1 - lag chunks only, so the plan -- and the arrangement of the result --
// depends on the input alone, not on timing.  Every position is written once:
// predecessors fill [0, t), successors [t, n).
#pragma once
#include <stdint.h>

#include <vector>

namespace lp {

struct HostPiece {
  uint64_t dev;   // first key on the device (index into the device copy)
  uint64_t host;  // first key in the host array
  uint64_t len;   // keys
};

class HostChunkPlan {
 public:
  void init(uint64_t n, uint64_t C, uint32_t lag) {
    n_ = n;
    C_ = C ? C : 1;
    lag_ = lag;
    K_ = (uint32_t)((n + C_ - 1) / C_);
    fnext_ = 0;
    bnext_ = (int64_t)K_ - 1;
    order_.clear();
    front_.clear();
    Fi_ = Bi_ = 0;
    P_ = S_ = 0;
    Pc_.assign(1, 0);
    Sc_.assign(1, 0);
    processed_ = 0;
    fdone_ = 0;
    bdone_ = n;
    pend_.clear();
  }
  uint32_t chunks() const { return K_; }
  uint64_t chunk_begin(uint32_t k) const { return (uint64_t)k * C_; }
  uint64_t chunk_len(uint32_t k) const {
    const uint64_t b = chunk_begin(k);
    return n_ - b < C_ ? n_ - b : C_;
  }
  uint32_t uploads() const { return (uint32_t)order_.size(); }
  uint32_t processed() const { return processed_; }
  // chunks whose counts the next upload's choice needs
  uint32_t needed_for_next() const {
    const int64_t m = (int64_t)order_.size() + 1 - (int64_t)lag_;
    return m > 0 ? (uint32_t)m : 0u;
  }
  // The chunk of the next upload; requires processed() >= needed_for_next()
  // and uploads() < chunks().
  uint32_t next_upload() {
    const uint32_t m = needed_for_next();
    const int64_t P = (int64_t)Pc_[m], S = (int64_t)Sc_[m];
    const int64_t U = (int64_t)(Fi_ + Bi_) - P - S;  // uploaded, counts not used
    const int64_t pf = 2 * P + U - 2 * (int64_t)Fi_;   // twice the front's waiting output
    const int64_t pb = 2 * S + U - 2 * (int64_t)Bi_;
    const bool front = fnext_ == (uint32_t)bnext_ || pf >= pb;
    const uint32_t k = front ? fnext_++ : (uint32_t)(bnext_--);
    order_.push_back(k);
    front_.push_back(front ? 1 : 0);
    (front ? Fi_ : Bi_) += chunk_len(k);
    return k;
  }
  // The next upload (in upload order) was partitioned on the device with p
  // predecessors; its upload is complete.  Returns false, changing nothing,
  // when there is no such upload or p exceeds the chunk's length (never a
  // valid split: no copy may be planned from it).
  bool partitioned(uint64_t p) {
    if (processed_ >= order_.size()) return false;
    if (p > chunk_len(order_[processed_])) return false;
    const uint32_t q = processed_++;
    const uint32_t k = order_[q];
    const uint64_t len = chunk_len(k), s = len - p, d0 = chunk_begin(k);
    if (p) pend_.push_back(Range{d0, P_, P_ + p, P_});
    if (s) pend_.push_back(Range{d0 + p, n_ - S_ - s, n_ - S_, n_ - S_ - s});
    P_ += p;
    S_ += s;
    Pc_.push_back(P_);
    Sc_.push_back(S_);
    if (front_[q]) {
      const uint64_t e = d0 + len;
      if (e > fdone_) fdone_ = e;
    } else if (d0 < bdone_) {
      bdone_ = d0;
    }
    return true;
  }
  // Appends the copies that became legal: host positions in [0, fdone) or
  // [bdone, n) have reached the device.
  void take_pieces(std::vector<HostPiece>& out) {
    size_t w = 0;
    for (size_t i = 0; i < pend_.size(); i++) {
      Range r = pend_[i];
      const uint64_t fe = r.r < fdone_ ? r.r : fdone_;
      if (r.l < fe) {
        out.push_back(HostPiece{r.dev + (r.l - r.dst0), r.l, fe - r.l});
        r.l = fe;
      }
      const uint64_t bb = r.l > bdone_ ? r.l : bdone_;
      if (bb < r.r) {
        out.push_back(HostPiece{r.dev + (bb - r.dst0), bb, r.r - bb});
        r.r = bb;
      }
      if (r.l < r.r) pend_[w++] = r;
    }
    pend_.resize(w);
  }
  uint64_t split() const { return P_; }
  bool finished() const { return processed_ == K_ && pend_.empty(); }

 private:
  struct Range {
    uint64_t dev;   // device key of host position dst0
    uint64_t l, r;  // host positions still to write
    uint64_t dst0;
  };
  uint64_t n_ = 0, C_ = 1;
  uint32_t lag_ = 0, K_ = 0;
  uint32_t fnext_ = 0;
  int64_t bnext_ = -1;
  std::vector<uint32_t> order_;
  std::vector<uint8_t> front_;
  uint64_t Fi_ = 0, Bi_ = 0;        // keys uploaded from the front / the back
  uint64_t P_ = 0, S_ = 0;          // predecessors / successors placed so far
  std::vector<uint64_t> Pc_, Sc_;   // ... after each processed chunk
  uint32_t processed_ = 0;
  uint64_t fdone_ = 0, bdone_ = 0;  // host [0, fdone) and [bdone, n) reached the device
  std::vector<Range> pend_;
};

}  // namespace lp
