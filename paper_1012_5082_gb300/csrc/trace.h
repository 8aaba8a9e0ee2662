// NVTX ranges around the library's public calls: a profiler that attaches
// (Nsight Systems, Nsight Compute's range filters) sees each call as a named
// range; without one a push or pop costs one function-pointer check.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace vcsgc {

struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace vcsgc

#define VCSGC_TRACE_CAT2(a, b) a##b
#define VCSGC_TRACE_CAT(a, b) VCSGC_TRACE_CAT2(a, b)
#define VCSGC_TRACE(name) ::vcsgc::TraceRange VCSGC_TRACE_CAT(vcsgc_trace_, __LINE__)(name)
