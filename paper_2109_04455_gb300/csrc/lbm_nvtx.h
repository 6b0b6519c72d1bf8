// NVTX range over one call of the C ABI (visible in profilers; a no-op
// without one).  Host code of the CUDA translation units only.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace lbm {

struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace lbm
