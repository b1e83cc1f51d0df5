// NVTX ranges (header-only NVTX v3) around the library's calls and passes,
// for profilers that follow them (ncu --nvtx, Nsight Systems).  With no tool
// attached a range costs one indirect call.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace afd_host {

class TraceRange {
public:
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace afd_host
