// Explicit instantiations of the forward kernels.  This file is compiled once
// per group of matrix sizes (-DPERM_PART=0..7) so the 48 x 3 kernels build in
// parallel.
#include "fwd_kernel.cuh"

#ifndef PERM_PART
#error "compile with -DPERM_PART=<0..7>"
#endif

// Instruction-mix variant used by the library (see TUNE in fwd_kernel.cuh).
#ifndef PERM_DEFAULT_TUNE
#define PERM_DEFAULT_TUNE 3
#endif

namespace permk {

template <int N, int PREC, int TUNE>
static int launch_one(const FwdArgs& a, int grid, int block, cudaStream_t s) {
  const size_t smem = fwd_smem_bytes(N, a.kind);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fwd_kernel<N, PREC, TUNE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fwd_smem_bytes(N, KIND_GLYNN));
    if (e != cudaSuccess) return (int)e;
  }
  fwd_kernel<N, PREC, TUNE><<<grid, block, smem, s>>>(a);
  return (int)cudaGetLastError();
}

template <int N, int PREC, int TUNE>
static int occupancy_one(int block, int kind, int* out) {
  const size_t smem = fwd_smem_bytes(N, kind);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fwd_kernel<N, PREC, TUNE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fwd_smem_bytes(N, KIND_GLYNN));
    if (e != cudaSuccess) return (int)e;
  }
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, fwd_kernel<N, PREC, TUNE>, block, smem);
}

// Sizes that also carry the four instruction-mix variants (for tuning runs).
template <int N>
struct HasTuneVariants {
  static constexpr bool value = (N == 24 || N == 32);
};

template <int N>
int launch_fwd(const FwdArgs& a, int prec, int tune, int grid, int block, cudaStream_t s) {
  if (prec == 1) return launch_one<N, 1, PERM_DEFAULT_TUNE>(a, grid, block, s);
  if (prec == 2) return launch_one<N, 2, PERM_DEFAULT_TUNE>(a, grid, block, s);
  if (prec == 3) return launch_one<N, 3, PERM_DEFAULT_TUNE>(a, grid, block, s);
  if (prec == 4) return launch_one<N, 4, PERM_DEFAULT_TUNE>(a, grid, block, s);
  if constexpr (HasTuneVariants<N>::value) {
    switch (tune) {
      case 0: return launch_one<N, 0, 0>(a, grid, block, s);
      case 1: return launch_one<N, 0, 1>(a, grid, block, s);
      case 2: return launch_one<N, 0, 2>(a, grid, block, s);
      case 3: return launch_one<N, 0, 3>(a, grid, block, s);
      default: break;
    }
  }
  return launch_one<N, 0, PERM_DEFAULT_TUNE>(a, grid, block, s);
}

template <int N>
int fwd_blocks_per_sm(int prec, int tune, int block, int kind, int* out) {
  if (prec == 1) return occupancy_one<N, 1, PERM_DEFAULT_TUNE>(block, kind, out);
  if (prec == 2) return occupancy_one<N, 2, PERM_DEFAULT_TUNE>(block, kind, out);
  if (prec == 3) return occupancy_one<N, 3, PERM_DEFAULT_TUNE>(block, kind, out);
  if (prec == 4) return occupancy_one<N, 4, PERM_DEFAULT_TUNE>(block, kind, out);
  if constexpr (HasTuneVariants<N>::value) {
    switch (tune) {
      case 0: return occupancy_one<N, 0, 0>(block, kind, out);
      case 1: return occupancy_one<N, 0, 1>(block, kind, out);
      case 2: return occupancy_one<N, 0, 2>(block, kind, out);
      case 3: return occupancy_one<N, 0, 3>(block, kind, out);
      default: break;
    }
  }
  return occupancy_one<N, 0, PERM_DEFAULT_TUNE>(block, kind, out);
}

#define PERM_INST(N)                                                                    \
  template int launch_fwd<N>(const FwdArgs&, int, int, int, int, cudaStream_t); \
  template int fwd_blocks_per_sm<N>(int, int, int, int, int*);

#if PERM_PART == 0
PERM_INST(1) PERM_INST(2) PERM_INST(3) PERM_INST(4) PERM_INST(5) PERM_INST(6)
PERM_INST(7) PERM_INST(8) PERM_INST(9) PERM_INST(10) PERM_INST(11) PERM_INST(12)
#elif PERM_PART == 1
PERM_INST(13) PERM_INST(14) PERM_INST(15) PERM_INST(16) PERM_INST(17) PERM_INST(18)
PERM_INST(19) PERM_INST(20)
#elif PERM_PART == 2
PERM_INST(21) PERM_INST(22) PERM_INST(23) PERM_INST(24) PERM_INST(25) PERM_INST(26)
#elif PERM_PART == 3
PERM_INST(27) PERM_INST(28) PERM_INST(29) PERM_INST(30) PERM_INST(31)
#elif PERM_PART == 4
PERM_INST(32) PERM_INST(33) PERM_INST(34) PERM_INST(35)
#elif PERM_PART == 5
PERM_INST(36) PERM_INST(37) PERM_INST(38) PERM_INST(39)
#elif PERM_PART == 6
PERM_INST(40) PERM_INST(41) PERM_INST(42) PERM_INST(43)
#elif PERM_PART == 7
PERM_INST(44) PERM_INST(45) PERM_INST(46) PERM_INST(47) PERM_INST(48)
#else
#error "PERM_PART out of range"
#endif

}  // namespace permk
