// lp_server.cu -- the serving engine (include/libpartition.h, "serving"):
// partition and sort requests of mixed sizes and key widths, admitted FIFO
// under a slot limit and a device-memory budget (lp_sched.h), and run by
// continuous batching: every engine step is one batched launch per key width
// that holds the newly admitted partition requests AND the current quicksort
// level of every sort in flight (lp_qs.cuh), followed by the children split
// and the shared-memory sorts of all those sorts.  Requests that arrive while
// a step runs join the next step; a partition finishes in the step it joins,
// a sort after as many steps as its quicksort has levels.
//
// A sort whose open subarrays are few and small (lp::qs_is_tail) finishes in
// its next step instead: one tail launch sorts each of them completely, one
// CTA per subarray.
//
// A request's result does not depend on what it was batched with: every
// segment's offsets X follow from the engine seed and the segment's own salt
// (the request seed, or a hash of the sort subarray), and the batched kernel
// treats segments independently.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <chrono>
#include <deque>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lp_batched.h"
#include "lp_ctx.h"
#include "lp_device.cuh"
#include "lp_qs.cuh"
#include "lp_sched.h"
#include "lp_trace.h"

namespace {

using lp::QsItem;
using lp::QsJob;
using lp::QsLevelCounts;
using lp::QsSmall;
using lp::SegDesc;

// Start of a sort's level: reset its level counts; a new sort also gets its
// first item (or, when small, its only small subarray).
struct QsBegin {
  QsLevelCounts* lc;
  QsItem* list0;
  QsSmall* small;
  uint64_t n;
  uint32_t mode;  // 0: next level, 1: new (one item), 2: new (small only)
  uint32_t pad;
};

// Adds the keys one batched launch streamed to the engine's total.
__global__ void add_traffic_kernel(const unsigned long long* traffic, unsigned long long* acc) {
  *acc += *traffic;
}

__global__ void qs_begin_kernel(const QsBegin* b, uint32_t count) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const QsBegin x = b[i];
  QsLevelCounts c{0u, 0u};
  if (x.mode == 1) x.list0[0] = QsItem{0, x.n, 0, 0};
  if (x.mode == 2) {
    x.small[0] = QsSmall{0, (uint32_t)x.n, 0u};
    c.small = 1u;
  }
  *x.lc = c;
}

enum : uint32_t { kQueued = 0, kActive = 1, kKept = 2 };

struct Req {
  uint64_t id = 0;
  lp_request r{};
  uint32_t state = kQueued;
  uint64_t off = 0;            // arena block: keys, then the sort's lists
  void* d_keys = nullptr;
  bool fresh = true;           // admitted, not yet in a step
  // sort state
  QsItem* lists[2] = {nullptr, nullptr};
  QsSmall* small = nullptr;
  uint32_t* merge = nullptr;   // the merge sort's indices into the small list
  uint32_t cur = 0, level = 0, slot = 0;
  uint64_t open = 0;
  uint64_t peak_open = 0;      // most open items any level of the sort held
  uint64_t max_next = 0;       // keys of its largest open item
  // result
  uint64_t split = 0;
  double admit_s = 0, done_s = 0;
  uint32_t steps = 0;
};

uint64_t max_items(uint64_t n) { return n / (lp::kQsCut + 1) + 1; }

uint64_t sort_list_bytes(uint64_t n) {
  if (n <= lp::kQsCut) return 0;
  return 2 * lp::Arena::rounded(max_items(n) * sizeof(QsItem)) +
         lp::Arena::rounded(2 * max_items(n) * sizeof(QsSmall)) +
         lp::Arena::rounded(2 * max_items(n) * sizeof(uint32_t));
}

uint64_t request_bytes(const lp_request& r) {
  const uint64_t keys = lp::Arena::rounded(r.n * (r.key_bits / 8));
  return keys + (r.kind == LP_REQ_SORT ? sort_list_bytes(r.n) : 0) +
         (r.kind == LP_REQ_SORT && r.n <= lp::kQsCut
              ? lp::Arena::rounded(sizeof(QsSmall)) + lp::Arena::rounded(sizeof(uint32_t))
              : 0);
}

// Device and pinned buffers of one key width.
struct WidthBufs {
  SegDesc* segs = nullptr;
  uint64_t* splits = nullptr;
  QsJob* jobs = nullptr;
  void* batch = nullptr;
  lp::BatchScratch B{};
};

}  // namespace

struct lp_server {
  lp_server_config cfg{};
  lp_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  std::chrono::steady_clock::time_point t0;
  std::string err;
  bool broken = false;
  // arena
  unsigned char* d_arena = nullptr;
  lp::Arena arena;
  // engine scratch
  void* d_engine = nullptr;
  WidthBufs w[2];                      // [0] uint64 keys, [1] uint32 keys
  QsLevelCounts* d_lc = nullptr;       // per slot
  unsigned long long* d_sorted = nullptr;  // per slot: keys sorted in shared memory
  unsigned long long* d_acc = nullptr;     // keys streamed by batched launches, per width
  cudaEvent_t ev[4] = {};                  // around each width's batched launch
  bool timed[2] = {false, false};
  QsBegin* d_begin = nullptr;
  uint32_t* d_ctl = nullptr;           // grid barrier (2 words), status
  unsigned long long* d_tail = nullptr;  // the tail kernels' tallies, 8 words per width
  uint32_t tail_grid[2] = {0, 0};        // CTAs of the tail kernel, per width
  // pinned staging
  unsigned char* h_stage = nullptr;
  size_t stage_bytes = 0;
  // requests
  uint64_t next_id = 1;
  std::unordered_map<uint64_t, Req> reqs;
  std::deque<uint64_t> queue;
  std::vector<uint64_t> active;
  std::vector<uint32_t> free_slots;
  std::vector<lp_completion> done;
  lp_server_stats stats{};
};

namespace {

double now_s(const lp_server* s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

lp_status srv_fail(lp_server* s, lp_status st, const std::string& what) {
  s->err = what;
  return st;
}

lp_status srv_cuda(lp_server* s, cudaError_t e, const char* where) {
  s->broken = true;
  return srv_fail(s, LP_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

size_t engine_bytes(uint32_t C, uint32_t slots) {
  size_t b = 0;
  for (int k = 0; k < 2; k++) {
    b += lp::Arena::rounded((size_t)C * sizeof(SegDesc)) + lp::Arena::rounded((size_t)C * 8) +
         lp::Arena::rounded((size_t)slots * sizeof(QsJob)) + lp::batch_scratch_bytes(C);
  }
  b += lp::Arena::rounded((size_t)slots * sizeof(QsLevelCounts)) +
       lp::Arena::rounded((size_t)slots * 8) + 256 +
       lp::Arena::rounded((size_t)slots * sizeof(QsBegin)) + 256 + 256;
  return b;
}

// pinned staging layout: jobs[2], partition records[2], begins, then read-back
struct Stage {
  QsJob* jobs[2];
  SegDesc* part[2];
  QsBegin* begin;
  QsLevelCounts* lc_back;
  uint64_t* split_back[2];
  uint32_t* status_back;
  size_t bytes;
};

Stage stage_layout(unsigned char* base, uint32_t slots) {
  Stage S{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* r = base ? base + off : nullptr;
    off += (bytes + 63) / 64 * 64;
    return r;
  };
  for (int k = 0; k < 2; k++) S.jobs[k] = reinterpret_cast<QsJob*>(take(slots * sizeof(QsJob)));
  for (int k = 0; k < 2; k++) S.part[k] = reinterpret_cast<SegDesc*>(take(slots * sizeof(SegDesc)));
  S.begin = reinterpret_cast<QsBegin*>(take(slots * sizeof(QsBegin)));
  S.lc_back = reinterpret_cast<QsLevelCounts*>(take(slots * sizeof(QsLevelCounts)));
  for (int k = 0; k < 2; k++) S.split_back[k] = reinterpret_cast<uint64_t*>(take(slots * 8));
  S.status_back = reinterpret_cast<uint32_t*>(take(64));
  S.bytes = off;
  return S;
}

void finish(lp_server* s, Req& q) {
  q.done_s = now_s(s);
  lp_completion c{};
  c.id = q.id;
  c.kind = q.r.kind;
  c.key_bits = q.r.key_bits;
  c.n = q.r.n;
  c.split = q.split;
  c.arrival_s = q.r.arrival_s;
  c.admit_s = q.admit_s;
  c.done_s = q.done_s;
  c.steps = q.steps;
  s->done.push_back(c);
  s->stats.completed++;
  s->stats.keys_done += q.r.n;
  if (q.r.kind == LP_REQ_SORT) s->free_slots.push_back(q.slot);
  if (s->cfg.keep_results) {
    q.state = kKept;
  } else {
    s->arena.release(q.off);
    s->reqs.erase(q.id);
  }
}

// Puts the request's keys in its arena block (stream-ordered before the step).
cudaError_t load_keys(lp_server* s, Req& q) {
  const uint64_t bytes = q.r.n * (q.r.key_bits / 8);
  if (q.r.n == 0) return cudaSuccess;
  if (q.r.d_src)
    return cudaMemcpyAsync(q.d_keys, q.r.d_src, bytes, cudaMemcpyDeviceToDevice, s->stream);
  if (q.r.key_bits == 64)
    return lp::launch_fill_u64(static_cast<uint64_t*>(q.d_keys), q.r.n, q.r.seed, s->stream);
  return lp::launch_fill_u32(static_cast<uint32_t*>(q.d_keys), q.r.n, q.r.seed, s->stream);
}

template <typename T>
cudaError_t run_width(lp_server* s, int k, uint32_t nparts, uint32_t njobs, uint32_t nsegs,
                      uint64_t max_open, uint64_t max_small) {
  WidthBufs& W = s->w[k];
  cudaStream_t st = s->stream;
  lp::LaunchCfg cfg{k == 0 ? s->ctx->grid_batch_u64 : s->ctx->grid_batch_u32, st, 0, nullptr};
  lp::BatchTuning tune{};
  tune.ctas = s->ctx->tuning.ctas;
  tune.line_bytes = s->ctx->tuning.line_bytes;
  tune.min_chunks = s->ctx->tuning.min_chunks;
  tune.group_workers = s->ctx->tuning.group_workers;
  tune.min_chunks_residual = s->ctx->tuning.min_chunks_residual;
  tune.mc_slices = s->ctx->tuning.onchip_slices;
  if (tune.ctas && tune.ctas < cfg.grid) cfg.grid = tune.ctas;
  cudaError_t e = cudaSuccess;
  if (njobs > 0 && max_open > 0) {
    if ((e = lp::launch_qs_build<T>(W.jobs, njobs, (uint32_t)max_open, W.segs, st)) != cudaSuccess)
      return e;
    cfg.launches++;
  }
  if (nsegs > 0) {
    if (s->ev[0] && (e = cudaEventRecord(s->ev[2 * k], st)) != cudaSuccess) return e;
    e = lp::launch_batched<T>(W.segs, nsegs, s->cfg.seed, W.splits, W.B, tune, cfg);
    if (e != cudaSuccess) return e;
    if (s->ev[0]) {
      if ((e = cudaEventRecord(s->ev[2 * k + 1], st)) != cudaSuccess) return e;
      s->timed[k] = true;
    }
    // children of the sorts' items; the keys this launch streamed go to the
    // engine's total
    if (njobs > 0 && max_open > 0) {
      e = lp::launch_qs_split(W.jobs, njobs, (uint32_t)max_open, W.segs, W.splits,
                              W.B.totals + 2, s->d_acc + k, st);
      if (e != cudaSuccess) return e;
    } else {
      add_traffic_kernel<<<1, 1, 0, st>>>(W.B.totals + 2, s->d_acc + k);
    }
    cfg.launches++;
  }
  if (njobs > 0 && max_small > 0) {
    e = lp::launch_qs_small_sort<T>(W.jobs, njobs,
                                    (uint32_t)(max_small < 2048 ? max_small : 2048), st);
    if (e != cudaSuccess) return e;
    cfg.launches++;
  }
  s->stats.launches += cfg.launches;
  (void)nparts;
  return cudaGetLastError();
}

lp_status engine_step(lp_server* s, uint32_t* in_flight) {
  const uint32_t slots = s->cfg.max_slots;
  const uint32_t C = s->cfg.max_segments;
  // ---- admission (FIFO, slots + budget)
  std::vector<uint64_t> adm(slots);
  auto fits = [&](uint64_t id) {
    Req& q = s->reqs[id];
    if (q.r.kind == LP_REQ_SORT && s->free_slots.empty()) return false;
    uint64_t off = 0;
    if (!s->arena.alloc(request_bytes(q.r), &off)) return false;
    q.off = off;
    return true;
  };
  const uint32_t room = slots > s->active.size() ? slots - (uint32_t)s->active.size() : 0;
  const uint32_t na = lp::admit_fifo(s->queue, room, fits, adm.data(), slots);
  const double t_adm = now_s(s);
  for (uint32_t i = 0; i < na; i++) {
    Req& q = s->reqs[adm[i]];
    q.state = kActive;
    q.admit_s = t_adm;
    q.d_keys = s->d_arena + q.off;
    if (q.r.kind == LP_REQ_SORT) {
      q.slot = s->free_slots.back();
      s->free_slots.pop_back();
      unsigned char* p = s->d_arena + q.off + lp::Arena::rounded(q.r.n * (q.r.key_bits / 8));
      if (q.r.n > lp::kQsCut) {
        const uint64_t m = max_items(q.r.n);
        q.lists[0] = reinterpret_cast<QsItem*>(p);
        q.lists[1] = reinterpret_cast<QsItem*>(p + lp::Arena::rounded(m * sizeof(QsItem)));
        q.small = reinterpret_cast<QsSmall*>(p + 2 * lp::Arena::rounded(m * sizeof(QsItem)));
        q.merge = reinterpret_cast<uint32_t*>(p + 2 * lp::Arena::rounded(m * sizeof(QsItem)) +
                                              lp::Arena::rounded(2 * m * sizeof(QsSmall)));
        q.open = 1;
        q.peak_open = 1;
        q.max_next = q.r.n;
      } else {
        q.small = reinterpret_cast<QsSmall*>(p);
        q.merge = reinterpret_cast<uint32_t*>(p + lp::Arena::rounded(sizeof(QsSmall)));
        q.open = 0;
      }
    }
    s->active.push_back(q.id);
    const uint64_t used = s->arena.used();
    if (used > s->stats.peak_bytes) s->stats.peak_bytes = used;
    cudaError_t e = load_keys(s, q);
    if (e != cudaSuccess) return srv_cuda(s, e, "load request keys");
  }
  // requests that need no device work finish at once
  for (size_t i = 0; i < s->active.size();) {
    Req& q = s->reqs[s->active[i]];
    const bool trivial = q.r.n < 2 ||
                         (q.r.kind == LP_REQ_PARTITION && q.r.n == 0);
    if (trivial && q.fresh) {
      if (q.r.kind == LP_REQ_PARTITION) {
        q.split = 0;
        if (q.r.n == 1) {
          // one key: the split is whether it is a predecessor; read it back
          uint64_t x = 0;
          cudaError_t e = cudaMemcpyAsync(&x, q.d_keys, q.r.key_bits / 8,
                                          cudaMemcpyDeviceToHost, s->stream);
          if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
          if (e != cudaSuccess) return srv_cuda(s, e, "read one key");
          q.split = x <= q.r.pivot ? 1 : 0;
        }
      }
      const uint64_t id = q.id;
      s->active.erase(s->active.begin() + i);
      finish(s, s->reqs[id]);
      continue;
    }
    i++;
  }
  if (s->active.empty()) {
    if (in_flight) *in_flight = 0;
    return LP_OK;
  }
  // ---- the step's tables, per key width
  Stage S = stage_layout(s->h_stage, slots);
  uint32_t nparts[2] = {0, 0}, njobs[2] = {0, 0}, nsegs[2] = {0, 0}, nbegin = 0;
  uint64_t max_open[2] = {0, 0}, max_small[2] = {0, 0};
  std::vector<uint64_t> part_ids[2], job_ids[2], tail_ids[2];
  for (uint64_t id : s->active) {  // partitions first: their records start each table
    Req& q = s->reqs[id];
    if (q.r.kind != LP_REQ_PARTITION) continue;
    const int k = q.r.key_bits == 64 ? 0 : 1;
    if (nsegs[k] + 1 > C) continue;  // waits for the next step
    SegDesc d{};
    d.keys = q.d_keys;
    d.n = q.r.n;
    d.pivot = q.r.pivot;
    d.salt = q.r.seed;
    S.part[k][nparts[k]++] = d;
    nsegs[k]++;
    part_ids[k].push_back(id);
  }
  for (uint64_t id : s->active) {
    Req& q = s->reqs[id];
    if (q.r.kind != LP_REQ_SORT) continue;
    const int k = q.r.key_bits == 64 ? 0 : 1;
    if (!q.fresh && lp::qs_is_tail(q.open, q.peak_open, q.max_next)) {
      tail_ids[k].push_back(id);  // the rest of the sort in this step, one CTA per item
      continue;
    }
    if (nsegs[k] + q.open > C) continue;  // the whole level or nothing; waits otherwise
    QsJob& J = S.jobs[k][njobs[k]++];
    J.keys = q.d_keys;
    J.items = q.lists[q.cur];
    J.next = q.lists[q.cur ^ 1];
    J.small = q.small;
    J.merge = q.merge;
    J.lc = s->d_lc + q.slot;
    J.sort_keys = s->d_sorted + q.slot;
    J.seed = q.r.seed;
    J.level = q.level;
    J.count = (uint32_t)q.open;
    J.seg_base = nsegs[k];
    J.samples = lp::kQsSamplesMax;  // median-of-15 pivots: fewer levels, lower latency
    J.local_cut = 0;                // small children: the shared-memory sort of each step
    nsegs[k] += (uint32_t)q.open;
    if (q.open > max_open[k]) max_open[k] = q.open;
    const uint64_t sb = q.open ? 2 * q.open : 1;
    if (sb > max_small[k]) max_small[k] = sb;
    QsBegin& b = S.begin[nbegin++];
    b.lc = J.lc;
    b.list0 = q.lists[0];
    b.small = q.small;
    b.n = q.r.n;
    b.mode = q.fresh ? (q.r.n > lp::kQsCut ? 1u : 2u) : 0u;
    b.pad = 0;
    job_ids[k].push_back(id);
  }
  // ---- upload and launch
  cudaStream_t st = s->stream;
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 2 && e == cudaSuccess; k++) {
    if (njobs[k])
      e = cudaMemcpyAsync(s->w[k].jobs, S.jobs[k], njobs[k] * sizeof(QsJob),
                          cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && nparts[k])
      e = cudaMemcpyAsync(s->w[k].segs, S.part[k], nparts[k] * sizeof(SegDesc),
                          cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess && nbegin) {
    e = cudaMemcpyAsync(s->d_begin, S.begin, nbegin * sizeof(QsBegin), cudaMemcpyHostToDevice,
                        st);
    if (e == cudaSuccess) {
      qs_begin_kernel<<<(nbegin + 255) / 256, 256, 0, st>>>(s->d_begin, nbegin);
      s->stats.launches++;
      e = cudaGetLastError();
    }
  }
  s->timed[0] = s->timed[1] = false;
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_ctl + 2, 0, 8, st);  // both status words
  if (e == cudaSuccess)
    e = run_width<uint64_t>(s, 0, nparts[0], njobs[0], nsegs[0], max_open[0], max_small[0]);
  if (e == cudaSuccess)
    e = run_width<uint32_t>(s, 1, nparts[1], njobs[1], nsegs[1], max_open[1], max_small[1]);
  // sorts in their tail: every open item sorted completely (median-of-15 pivots,
  // as in the levels)
  for (int k = 0; k < 2 && e == cudaSuccess; k++) {
    for (uint64_t id : tail_ids[k]) {
      Req& q = s->reqs[id];
      e = k == 0 ? lp::launch_qs_local<uint64_t>(static_cast<uint64_t*>(q.d_keys),
                                                 q.lists[q.cur], (uint32_t)q.open, q.level,
                                                 q.r.seed, lp::kQsSamplesMax, s->d_tail,
                                                 s->d_ctl + 2, s->tail_grid[0], st)
                 : lp::launch_qs_local<uint32_t>(static_cast<uint32_t*>(q.d_keys),
                                                 q.lists[q.cur], (uint32_t)q.open, q.level,
                                                 q.r.seed, lp::kQsSamplesMax, s->d_tail + 8,
                                                 s->d_ctl + 3, s->tail_grid[1], st);
      if (e != cudaSuccess) break;
      s->stats.launches += 2;
    }
  }
  // ---- read back: level counts of every slot, partition splits, status
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(S.lc_back, s->d_lc, slots * sizeof(QsLevelCounts),
                        cudaMemcpyDeviceToHost, st);
  for (int k = 0; k < 2 && e == cudaSuccess; k++)
    if (nparts[k])
      e = cudaMemcpyAsync(S.split_back[k], s->w[k].splits, nparts[k] * 8,
                          cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(S.status_back, s->d_ctl + 2, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return srv_cuda(s, e, "engine step");
  const uint32_t dev_status = S.status_back[0] | S.status_back[1];
  if (dev_status != 0) {
    s->broken = true;
    const bool timeout = (dev_status & lp::kStatTimeout) != 0;
    return srv_fail(s, timeout ? LP_ERR_TIMEOUT : LP_ERR_INTERNAL,
                    timeout ? lp_timeout_what(dev_status) : "device status after an engine step");
  }
  // small subarrays the bucket sort turned down: merge sorted before any
  // result counts as done or any list is reused
  bool merged = false;
  for (int k = 0; k < 2 && e == cudaSuccess; k++) {
    uint32_t most = 0;
    for (uint64_t id : job_ids[k]) {
      const uint32_t m = S.lc_back[s->reqs[id].slot].merge;
      most = m > most ? m : most;
    }
    if (most == 0) continue;
    const uint32_t ctas = most < 2048 ? most : 2048;
    e = k == 0 ? lp::launch_qs_merge_sort<uint64_t>(s->w[0].jobs, njobs[0], ctas, st)
               : lp::launch_qs_merge_sort<uint32_t>(s->w[1].jobs, njobs[1], ctas, st);
    s->stats.launches++;
    merged = true;
  }
  if (e == cudaSuccess && merged) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return srv_cuda(s, e, "merge sort");
  s->stats.steps++;
  for (int k = 0; k < 2; k++) {
    float ms = 0.f;
    if (s->timed[k] && cudaEventElapsedTime(&ms, s->ev[2 * k], s->ev[2 * k + 1]) == cudaSuccess)
      s->stats.batched_ms += ms;
  }
  // ---- outcomes
  std::vector<uint64_t> finished;
  for (int k = 0; k < 2; k++) {
    for (uint32_t i = 0; i < part_ids[k].size(); i++) {
      Req& q = s->reqs[part_ids[k][i]];
      q.split = S.split_back[k][i];
      q.steps++;
      q.fresh = false;
      finished.push_back(q.id);
    }
    for (uint64_t id : job_ids[k]) {
      Req& q = s->reqs[id];
      q.steps++;
      q.fresh = false;
      if (q.open == 0) {  // the small-only sort ran this step
        finished.push_back(id);
        continue;
      }
      q.level++;
      q.cur ^= 1;
      q.open = S.lc_back[q.slot].next;
      q.max_next = S.lc_back[q.slot].max_next;
      if (q.open > q.peak_open) q.peak_open = q.open;
      if (q.open == 0) finished.push_back(id);
    }
    for (uint64_t id : tail_ids[k]) {  // sorted completely this step
      Req& q = s->reqs[id];
      q.steps++;
      finished.push_back(id);
    }
  }
  for (uint64_t id : finished) {
    for (size_t i = 0; i < s->active.size(); i++)
      if (s->active[i] == id) {
        s->active.erase(s->active.begin() + i);
        break;
      }
    finish(s, s->reqs[id]);
  }
  if (in_flight) *in_flight = (uint32_t)s->active.size();
  return LP_OK;
}

lp_status check_request(lp_server* s, const lp_request* r) {
  if (!r) return srv_fail(s, LP_ERR_INVALID_ARG, "null request");
  if (r->kind != LP_REQ_PARTITION && r->kind != LP_REQ_SORT)
    return srv_fail(s, LP_ERR_INVALID_ARG, "unknown request kind");
  if (r->key_bits != 32 && r->key_bits != 64)
    return srv_fail(s, LP_ERR_INVALID_ARG, "key_bits must be 32 or 64");
  if (r->d_src && (reinterpret_cast<uintptr_t>(r->d_src) % (r->key_bits / 8)))
    return srv_fail(s, LP_ERR_INVALID_ARG, "d_src not aligned");
  if (request_bytes(*r) > s->arena.capacity())
    return srv_fail(s, LP_ERR_INVALID_ARG, "request larger than the budget");
  if (r->kind == LP_REQ_SORT && max_items(r->n) > s->cfg.max_segments)
    return srv_fail(s, LP_ERR_INVALID_ARG, "sort larger than one step can hold");
  return LP_OK;
}

// One request at a time through the plain calls, in arrival order.
lp_status run_one_at_a_time(lp_server* s, const lp_request* reqs, uint32_t count, double t0,
                            lp_completion* out) {
  for (uint32_t i = 0; i < count; i++) {
    const lp_request& r = reqs[i];
    lp_status st = check_request(s, &r);
    if (st != LP_OK) return st;
    while (now_s(s) < t0 + r.arrival_s) std::this_thread::yield();
    Req q;
    q.id = s->next_id++;
    q.r = r;
    q.r.arrival_s = t0 + r.arrival_s;
    uint64_t off = 0;
    if (!s->arena.alloc(request_bytes(r), &off))
      return srv_fail(s, LP_ERR_OOM, "request does not fit the budget");
    q.off = off;
    q.d_keys = s->d_arena + off;
    q.admit_s = now_s(s);
    cudaError_t e = load_keys(s, q);
    if (e != cudaSuccess) return srv_cuda(s, e, "load request keys");
    uint64_t t = 0;
    if (r.kind == LP_REQ_PARTITION) {
      st = r.key_bits == 64
               ? lp_partition_u64(s->ctx, static_cast<uint64_t*>(q.d_keys), r.n, r.pivot,
                                  LP_SMOOTHED, r.seed, s->stream, &t)
               : lp_partition_u32(s->ctx, static_cast<uint32_t*>(q.d_keys), r.n,
                                  (uint32_t)r.pivot, LP_SMOOTHED, r.seed, s->stream, &t);
    } else {
      st = r.key_bits == 64
               ? lp_quicksort_u64(s->ctx, static_cast<uint64_t*>(q.d_keys), r.n, r.seed,
                                  s->stream)
               : lp_quicksort_u32(s->ctx, static_cast<uint32_t*>(q.d_keys), r.n, r.seed,
                                  s->stream);
      if (st == LP_OK && cudaStreamSynchronize(s->stream) != cudaSuccess) st = LP_ERR_CUDA;
    }
    if (st != LP_OK) return srv_fail(s, st, lp_ctx_last_error(s->ctx));
    s->stats.launches += lp_ctx_last_launches(s->ctx);
    q.split = t;
    q.steps = 1;
    q.done_s = now_s(s);
    s->arena.release(off);
    lp_completion& c = out[i];
    c = lp_completion{};
    c.id = q.id;
    c.kind = r.kind;
    c.key_bits = r.key_bits;
    c.n = r.n;
    c.split = t;
    c.arrival_s = q.r.arrival_s;
    c.admit_s = q.admit_s;
    c.done_s = q.done_s;
    c.steps = 1;
    s->stats.completed++;
    s->stats.keys_done += r.n;
  }
  return LP_OK;
}

}  // namespace

extern "C" {

lp_status lp_server_create(int device, const lp_server_config* cfg, lp_server** out) {
  if (!cfg || !out) return LP_ERR_INVALID_ARG;
  *out = nullptr;
  lp_server* s = new lp_server();
  s->cfg = *cfg;
  if (!s->cfg.max_slots) s->cfg.max_slots = 256;
  if (!s->cfg.max_segments) s->cfg.max_segments = 65536;
  s->t0 = std::chrono::steady_clock::now();
  auto fail = [&](lp_status st) {
    lp_server_destroy(s);
    return st;
  };
  if (lp_ctx_create(&s->ctx, device) != LP_OK) return fail(LP_ERR_CUDA);
  if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail(LP_ERR_CUDA);
  const uint64_t cap = s->cfg.budget_bytes / lp::Arena::kArenaAlign * lp::Arena::kArenaAlign;
  if (cap == 0) return fail(LP_ERR_INVALID_ARG);
  if (cudaMalloc(&s->d_arena, cap) != cudaSuccess) return fail(LP_ERR_OOM);
  s->arena.reset(cap);
  const uint32_t C = s->cfg.max_segments, slots = s->cfg.max_slots;
  if (cudaMalloc(&s->d_engine, engine_bytes(C, slots)) != cudaSuccess) return fail(LP_ERR_OOM);
  unsigned char* p = static_cast<unsigned char*>(s->d_engine);
  auto take = [&](size_t bytes) {
    unsigned char* r = p;
    p += lp::Arena::rounded(bytes);
    return r;
  };
  for (int k = 0; k < 2; k++) {
    s->w[k].segs = reinterpret_cast<SegDesc*>(take((size_t)C * sizeof(SegDesc)));
    s->w[k].splits = reinterpret_cast<uint64_t*>(take((size_t)C * 8));
    s->w[k].jobs = reinterpret_cast<QsJob*>(take((size_t)slots * sizeof(QsJob)));
    s->w[k].batch = take(lp::batch_scratch_bytes(C));
  }
  s->d_lc = reinterpret_cast<QsLevelCounts*>(take((size_t)slots * sizeof(QsLevelCounts)));
  s->d_sorted = reinterpret_cast<unsigned long long*>(take((size_t)slots * 8));
  s->d_acc = reinterpret_cast<unsigned long long*>(take(256));
  s->d_begin = reinterpret_cast<QsBegin*>(take((size_t)slots * sizeof(QsBegin)));
  s->d_ctl = reinterpret_cast<uint32_t*>(take(256));
  s->d_tail = reinterpret_cast<unsigned long long*>(take(256));
  if (lp::qs_local_grid<uint64_t>(device, &s->tail_grid[0]) != cudaSuccess ||
      lp::qs_local_grid<uint32_t>(device, &s->tail_grid[1]) != cudaSuccess)
    return fail(LP_ERR_CUDA);
  // the batched launches of both widths share the barrier and status words
  // the batched launches of both widths share the barrier words; each has
  // its own status word (a launch resets its own)
  for (int k = 0; k < 2; k++)
    s->w[k].B = lp::carve_batch_scratch(s->w[k].batch, C, s->d_ctl, s->d_ctl + 2 + k);
  if (cudaMemset(s->d_engine, 0, engine_bytes(C, slots)) != cudaSuccess) return fail(LP_ERR_CUDA);
  s->stage_bytes = stage_layout(nullptr, slots).bytes;
  if (cudaMallocHost(&s->h_stage, s->stage_bytes) != cudaSuccess) return fail(LP_ERR_OOM);
  for (uint32_t i = 0; i < slots; i++) s->free_slots.push_back(slots - 1 - i);
  if (s->cfg.timing)
    for (int i = 0; i < 4; i++)
      if (cudaEventCreate(&s->ev[i]) != cudaSuccess) return fail(LP_ERR_CUDA);
  s->stats.engine_bytes = engine_bytes(C, slots);
  *out = s;
  return LP_OK;
}

lp_status lp_server_destroy(lp_server* s) {
  if (!s) return LP_ERR_INVALID_ARG;
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (int i = 0; i < 4; i++)
    if (s->ev[i]) cudaEventDestroy(s->ev[i]);
  if (s->h_stage) cudaFreeHost(s->h_stage);
  if (s->d_engine) cudaFree(s->d_engine);
  if (s->d_arena) cudaFree(s->d_arena);
  if (s->stream) cudaStreamDestroy(s->stream);
  if (s->ctx) lp_ctx_destroy(s->ctx);
  delete s;
  return LP_OK;
}

const char* lp_server_last_error(const lp_server* s) { return s ? s->err.c_str() : "null server"; }

double lp_server_now(const lp_server* s) { return s ? now_s(s) : 0.0; }

lp_status lp_server_submit(lp_server* s, const lp_request* r, uint64_t* id_out) {
  if (!s) return LP_ERR_INVALID_ARG;
  lp_status st = check_request(s, r);
  if (st != LP_OK) return st;
  Req q;
  q.id = s->next_id++;
  q.r = *r;
  s->reqs[q.id] = q;
  s->queue.push_back(q.id);
  if (id_out) *id_out = q.id;
  return LP_OK;
}

lp_status lp_server_step(lp_server* s, uint32_t* in_flight) {
  LP_TRACE("lp_server_step");
  if (!s) return LP_ERR_INVALID_ARG;
  if (s->broken) return srv_fail(s, LP_ERR_CUDA, "server stopped after an error");
  cudaError_t e = cudaSetDevice(s->ctx->device);
  if (e != cudaSuccess) return srv_cuda(s, e, "cudaSetDevice");
  const double t = now_s(s);
  lp_status st = engine_step(s, in_flight);
  s->stats.busy_s += now_s(s) - t;
  return st;
}

lp_status lp_server_poll(lp_server* s, lp_completion* out, uint32_t cap, uint32_t* got) {
  if (!s || !got || (cap && !out)) return LP_ERR_INVALID_ARG;
  const uint32_t k = (uint32_t)(s->done.size() < cap ? s->done.size() : cap);
  for (uint32_t i = 0; i < k; i++) out[i] = s->done[i];
  s->done.erase(s->done.begin(), s->done.begin() + k);
  *got = k;
  return LP_OK;
}

lp_status lp_server_result(lp_server* s, uint64_t id, void** d_keys) {
  if (!s || !d_keys) return LP_ERR_INVALID_ARG;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end() || it->second.state != kKept)
    return srv_fail(s, LP_ERR_INVALID_ARG, "no kept result with this id");
  *d_keys = it->second.d_keys;
  return LP_OK;
}

lp_status lp_server_fetch(lp_server* s, uint64_t id, void* dst, uint64_t bytes) {
  if (!s || (bytes && !dst)) return LP_ERR_INVALID_ARG;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end() || it->second.state != kKept)
    return srv_fail(s, LP_ERR_INVALID_ARG, "no kept result with this id");
  const Req& q = it->second;
  if (bytes > q.r.n * (q.r.key_bits / 8))
    return srv_fail(s, LP_ERR_INVALID_ARG, "more bytes than the request holds");
  cudaError_t e = cudaMemcpyAsync(dst, q.d_keys, bytes, cudaMemcpyDefault, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return srv_cuda(s, e, "fetch result");
  return LP_OK;
}

lp_status lp_server_release(lp_server* s, uint64_t id) {
  if (!s) return LP_ERR_INVALID_ARG;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end() || it->second.state != kKept)
    return srv_fail(s, LP_ERR_INVALID_ARG, "no kept result with this id");
  s->arena.release(it->second.off);
  s->reqs.erase(it);
  return LP_OK;
}

lp_status lp_server_get_stats(const lp_server* s, lp_server_stats* out) {
  if (!s || !out) return LP_ERR_INVALID_ARG;
  *out = s->stats;
  out->budget_bytes = s->arena.capacity();
  out->in_use_bytes = s->arena.used();
  return LP_OK;
}

lp_status lp_server_streamed_keys(lp_server* s, uint64_t* keys_u64, uint64_t* keys_u32) {
  if (!s || !keys_u64 || !keys_u32) return LP_ERR_INVALID_ARG;
  unsigned long long v[2] = {0, 0};
  cudaError_t e = cudaMemcpyAsync(s->h_stage, s->d_acc, 16, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return srv_cuda(s, e, "read streamed keys");
  memcpy(v, s->h_stage, 16);
  *keys_u64 = v[0];
  *keys_u32 = v[1];
  return LP_OK;
}

lp_status lp_server_run(lp_server* s, const lp_request* reqs, uint32_t count, uint32_t mode,
                        lp_completion* out) {
  LP_TRACE("lp_server_run");
  if (!s || (count && (!reqs || !out))) return LP_ERR_INVALID_ARG;
  if (s->broken) return srv_fail(s, LP_ERR_CUDA, "server stopped after an error");
  cudaError_t e = cudaSetDevice(s->ctx->device);
  if (e != cudaSuccess) return srv_cuda(s, e, "cudaSetDevice");
  for (uint32_t i = 1; i < count; i++)
    if (reqs[i].arrival_s < reqs[i - 1].arrival_s)
      return srv_fail(s, LP_ERR_INVALID_ARG, "arrivals must be in time order");
  const double t0 = now_s(s);
  if (mode == LP_SERVE_ONE_AT_A_TIME) {
    lp_status st = run_one_at_a_time(s, reqs, count, t0, out);
    s->stats.busy_s += now_s(s) - t0;
    return st;
  }
  if (mode != LP_SERVE_CONTINUOUS) return srv_fail(s, LP_ERR_INVALID_ARG, "unknown mode");
  // request i gets id first + i
  const uint64_t first = s->next_id;
  uint32_t next = 0, got = 0;
  std::vector<lp_completion> buf(256);
  while (got < count) {
    const double t = now_s(s) - t0;
    while (next < count && reqs[next].arrival_s <= t) {
      lp_request r = reqs[next];
      r.arrival_s = t0 + r.arrival_s;
      lp_status st = lp_server_submit(s, &r, nullptr);
      if (st != LP_OK) return st;
      next++;
    }
    if (s->active.empty() && s->queue.empty()) {
      std::this_thread::yield();  // idle until the next arrival
      continue;
    }
    uint32_t inflight = 0;
    lp_status st = lp_server_step(s, &inflight);
    if (st != LP_OK) return st;
    uint32_t k = 0;
    do {
      lp_server_poll(s, buf.data(), (uint32_t)buf.size(), &k);
      for (uint32_t i = 0; i < k; i++) {
        const uint64_t idx = buf[i].id - first;
        if (idx < count) {  // (completions of requests submitted elsewhere are dropped)
          out[idx] = buf[i];
          got++;
        }
      }
    } while (k == buf.size());
  }
  return LP_OK;
}

}  // extern "C"
