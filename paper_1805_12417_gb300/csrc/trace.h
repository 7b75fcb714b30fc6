// NVTX ranges around the host-side phases of a solve (whole call, outer
// step, inner CG solve), so a profiler's timeline (ncu --nvtx, Nsight
// Systems) can attribute kernels to them.  NVTX v3 is header-only: with no
// tool attached every call returns at once.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace mrcg {

struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace mrcg
