// lp_trace.h -- NVTX ranges around the library's entry points: each call
// shows as a named span in a profiler's timeline (Nsight Systems, ncu's NVTX
// filters).  NVTX3 is header-only; with no profiler attached a range costs
// one indirect call to a no-op.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace lp {

class TraceRange {
 public:
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace lp

// a range named `name` from here to the end of the enclosing scope
#define LP_TRACE(name) ::lp::TraceRange lp_trace_range_(name)
