// lbm_trace.h -- NVTX ranges around the library's host-visible phases (set-up, steps,
// transfers, reductions, pool chunks), so that a timeline profiler shows where a caller's
// time goes.  NVTX3 is header-only: with no profiler attached a range costs a branch.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace lbm {

class NvtxRange {
  public:
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace lbm

#define LBM_NVTX_CAT2(a, b) a##b
#define LBM_NVTX_CAT(a, b) LBM_NVTX_CAT2(a, b)
#define LBM_NVTX_RANGE(name) ::lbm::NvtxRange LBM_NVTX_CAT(lbm_nvtx_range_, __LINE__)(name)
