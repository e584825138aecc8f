// trace.h -- NVTX ranges around the public entry points, so that a
// profiler's timeline (Nsight Systems) shows each library call on the host
// thread that made it.  NVTX v3 is header-only; with no profiler attached a
// range costs a pointer check.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace sincos_gb300 {

struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace sincos_gb300

#define SINCOS_TRACE(name) ::sincos_gb300::TraceRange sincos_trace_range_(name)
