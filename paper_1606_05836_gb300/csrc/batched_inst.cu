// Instantiation of the persistent batched walk kernel for one precision rung
// (compiled once per rung with -DPERM_PREC=0..4 so the rungs build in parallel).
#include "batched_kernel.cuh"

#ifndef PERM_PREC
#error "compile with -DPERM_PREC=<0..4>"
#endif

namespace permk {

template <int PREC>
int launch_batch_walk(const BatchArgs& a, int grid, int block, cudaStream_t s) {
  batch_walk_kernel<PREC, 3><<<grid, block, 0, s>>>(a);
  return (int)cudaGetLastError();
}

template <int PREC>
int batch_walk_blocks_per_sm(int block, int* out) {
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, batch_walk_kernel<PREC, 3>, block, 0);
}

template int launch_batch_walk<PERM_PREC>(const BatchArgs&, int, int, cudaStream_t);
template int batch_walk_blocks_per_sm<PERM_PREC>(int, int*);

}  // namespace permk
