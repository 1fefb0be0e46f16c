// pa_trace.h -- NVTX ranges around the library's host entry points, so that a
// timeline profiler shows its phases (resampling, sweeps, observables, whole
// runs, checkpoints, the batched engine, the multi-GPU exchange steps) by
// name.  NVTX 3 is header-only; with no profiler attached a range costs a
// check of a function pointer.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace pa {

class TraceRange {
  public:
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace pa
