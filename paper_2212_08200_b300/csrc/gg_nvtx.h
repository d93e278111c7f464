// gg_nvtx.h -- an NVTX range around one public call of the C ABI.
//
// NVTX3 is header-only: without a profiler attached each push / pop is a
// call through an uninitialised function pointer that returns at once.  With
// one attached, a profile can select the launches of one call by its range.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace gg {

struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace gg
