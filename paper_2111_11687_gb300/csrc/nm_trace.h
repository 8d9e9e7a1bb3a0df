// NVTX ranges over the library's host calls, so that a profiler can group or
// filter the kernels a call launches by the call's name (for example
// `ncu --nvtx --nvtx-include "nm_dose_run/"`, or a timeline tool).  NVTX v3 is
// header-only: without an attached tool each push and pop returns at once.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace nm {

class NvtxRange {
 public:
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace nm
