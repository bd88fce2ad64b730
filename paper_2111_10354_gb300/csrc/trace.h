// NVTX ranges around solver phases, for Nsight tools (NVTX 3 is header-only: without a tool
// attached a range costs one check of a function pointer).
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace hisq {

struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace hisq
