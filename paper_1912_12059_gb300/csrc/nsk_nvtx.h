// nsk_nvtx.h -- NVTX ranges around the library's public calls (timeline annotation for profilers
// such as Nsight Systems). NVTX3 is header-only: without a profiler attached each range is a
// pair of cheap no-op calls.
#pragma once

#include <nvtx3/nvToolsExt.h>

struct NskRange {
  explicit NskRange(const char* name) { nvtxRangePushA(name); }
  ~NskRange() { nvtxRangePop(); }
  NskRange(const NskRange&) = delete;
  NskRange& operator=(const NskRange&) = delete;
};
