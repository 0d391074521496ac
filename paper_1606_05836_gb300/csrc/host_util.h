// Host-side helpers shared by the C ABI translation units.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace permk {
// NVTX range around one C-ABI call (visible in Nsight timelines; a no-op without a tool).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Records the cudaError_t reported by perm_last_cuda_error() on this thread.
void record_cuda_error(int err);
}  // namespace permk
