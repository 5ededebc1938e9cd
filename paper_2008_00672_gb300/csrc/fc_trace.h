// Host-side tracing of the ABI calls (no kernel includes this file).
#pragma once

#include <nvtx3/nvToolsExt.h>

// An NVTX range over one ABI call, named after the call: visible on profiler timelines
// and usable as an ncu/nsys filter; without a tool attached each push/pop is a no-op.
struct FcRange {
  explicit FcRange(const char* name) { nvtxRangePushA(name); }
  ~FcRange() { nvtxRangePop(); }
  FcRange(const FcRange&) = delete;
  FcRange& operator=(const FcRange&) = delete;
};
