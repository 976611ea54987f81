// NVTX ranges around the C entry points, named after the entry point, so
// that Nsight Systems timelines and ncu's NVTX range filters see each call.
// NVTX 3 is header-only and resolves its tool at run time: with no tool
// attached a range costs a few nanoseconds.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace spg {
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};
}  // namespace spg

#define SPG_TRACE() const spg::TraceRange spg_trace_range_(__func__)
