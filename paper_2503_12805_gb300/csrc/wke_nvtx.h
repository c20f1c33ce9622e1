// NVTX ranges around the library's calls: a profiler (Nsight Systems, ncu's
// range filters) shows them on its timeline; without a tool attached a range
// costs two calls into the header-only NVTX stubs.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace wke {

// An NVTX range for the lifetime of the object.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace wke
