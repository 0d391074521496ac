// Host-side helpers shared by the C ABI translation units.
#pragma once

namespace permk {
// Records the cudaError_t reported by perm_last_cuda_error() on this thread.
void record_cuda_error(int err);
}  // namespace permk
