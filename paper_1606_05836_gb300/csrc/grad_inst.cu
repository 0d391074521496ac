// Explicit instantiations of the adjoint kernel, compiled once per group of
// sizes (-DPERM_PART=0..3).
#include "grad_kernel.cuh"

#ifndef PERM_PART
#error "compile with -DPERM_PART=<0..3>"
#endif

namespace permk {

template <int N, int PREC>
static int launch_one(const GradArgs& a, int grid, cudaStream_t s) {
  const size_t smem = grad_smem_bytes(N);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(grad_kernel<N, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
  }
  grad_kernel<N, PREC><<<grid, GRAD_BLOCK, smem, s>>>(a);
  return (int)cudaGetLastError();
}

template <int N, int PREC>
static int occupancy_one(int* out) {
  const size_t smem = grad_smem_bytes(N);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(grad_kernel<N, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
  }
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, grad_kernel<N, PREC>, GRAD_BLOCK, smem);
}

// prec: 0 = FP64 (PERM_FP64), 3 = double-float products (PERM_FP64_DF)
template <int N>
int launch_grad(const GradArgs& a, int prec, int grid, cudaStream_t s) {
  return prec == 3 ? launch_one<N, 3>(a, grid, s) : launch_one<N, 0>(a, grid, s);
}

template <int N>
int grad_blocks_per_sm(int prec, int* out) {
  return prec == 3 ? occupancy_one<N, 3>(out) : occupancy_one<N, 0>(out);
}

#define PERM_GINST(N)                                                        \
  template int launch_grad<N>(const GradArgs&, int, int, cudaStream_t); \
  template int grad_blocks_per_sm<N>(int, int*);

#if PERM_PART == 0
PERM_GINST(1) PERM_GINST(2) PERM_GINST(3) PERM_GINST(4) PERM_GINST(5) PERM_GINST(6) PERM_GINST(7) PERM_GINST(8)
PERM_GINST(9) PERM_GINST(10) PERM_GINST(11) PERM_GINST(12) PERM_GINST(13) PERM_GINST(14)
#elif PERM_PART == 1
PERM_GINST(15) PERM_GINST(16) PERM_GINST(17) PERM_GINST(18) PERM_GINST(19) PERM_GINST(20) PERM_GINST(21)
#elif PERM_PART == 2
PERM_GINST(22) PERM_GINST(23) PERM_GINST(24) PERM_GINST(25) PERM_GINST(26) PERM_GINST(27)
#elif PERM_PART == 3
PERM_GINST(28) PERM_GINST(29) PERM_GINST(30) PERM_GINST(31) PERM_GINST(32)
#else
#error "PERM_PART out of range"
#endif

}  // namespace permk
