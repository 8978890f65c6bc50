// NVTX ranges around the library's entry points (tracing: a profiler that
// is attached sees every emc_* call as a named range over its launches; with
// no tool attached NVTX does nothing).  Header-only NVTX 3.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace emc {
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};
}  // namespace emc

#define EMC_TRACE(name) ::emc::TraceRange emc_trace_range_(name)
