// nvtx_range.h -- NVTX ranges around the library's host-side operations
// (plan creation, transforms, batches, tuning, serving), so that a profiler
// timeline (Nsight Systems, or ncu --nvtx filters) shows which library call
// issued which kernels.  NVTX v3 is header-only: without a tool attached the
// push/pop calls return at once.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace gb300ntt {

class NvtxRange {
 public:
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace gb300ntt
