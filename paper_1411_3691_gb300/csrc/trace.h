// trace.h -- NVTX ranges around the host side of the entry points (plan, launches, reduce),
// so a profiler's timeline shows where each call spends its time.  NVTX v3 is header-only:
// without a tool attached a range costs two calls into a stub.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace mhc {

struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace mhc
