// Explicit instantiations of the row-minor kernel (FP64, R3 and R4), compiled
// once per group of sizes (-DPERM_PART=0..3).
#include "minors_kernel.cuh"

#ifndef PERM_PART
#error "compile with -DPERM_PART=<0..1>"
#endif

namespace permk {

template <int K, int PREC>
static int minors_smem_attr() {
  const size_t smem = minors_smem_bytes(K);
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(minors_kernel<K, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
  }
  return 0;
}

template <int K, int PREC>
static int launch_one_minors(const MinorsArgs& a, int grid, cudaStream_t s) {
  int e = minors_smem_attr<K, PREC>();
  if (e) return e;
  minors_kernel<K, PREC><<<grid, MINORS_BLOCK, minors_smem_bytes(K), s>>>(a);
  return (int)cudaGetLastError();
}

template <int K, int PREC>
static int occupancy_one_minors(int* out) {
  int e = minors_smem_attr<K, PREC>();
  if (e) return e;
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, minors_kernel<K, PREC>, MINORS_BLOCK,
                                                            minors_smem_bytes(K));
}

template <int K>
int launch_minors(const MinorsArgs& a, int prec, int grid, cudaStream_t s) {
  if (prec == 4) return launch_one_minors<K, 4>(a, grid, s);
  if (prec == 3) return launch_one_minors<K, 3>(a, grid, s);
  return launch_one_minors<K, 0>(a, grid, s);
}

template <int K>
int minors_blocks_per_sm(int prec, int* out) {
  if (prec == 4) return occupancy_one_minors<K, 4>(out);
  if (prec == 3) return occupancy_one_minors<K, 3>(out);
  return occupancy_one_minors<K, 0>(out);
}

#define PERM_MINST(K)                                                       \
  template int launch_minors<K>(const MinorsArgs&, int, int, cudaStream_t); \
  template int minors_blocks_per_sm<K>(int, int*);

#if PERM_PART == 0
PERM_MINST(2) PERM_MINST(3) PERM_MINST(4) PERM_MINST(5) PERM_MINST(6) PERM_MINST(7) PERM_MINST(8) PERM_MINST(9)
PERM_MINST(10) PERM_MINST(11) PERM_MINST(12) PERM_MINST(13) PERM_MINST(14) PERM_MINST(15) PERM_MINST(16)
#elif PERM_PART == 1
PERM_MINST(17) PERM_MINST(18) PERM_MINST(19) PERM_MINST(20) PERM_MINST(21) PERM_MINST(22)
#elif PERM_PART == 2
PERM_MINST(23) PERM_MINST(24) PERM_MINST(25) PERM_MINST(26) PERM_MINST(27)
#elif PERM_PART == 3
PERM_MINST(28) PERM_MINST(29) PERM_MINST(30) PERM_MINST(31) PERM_MINST(32)
#else
#error "PERM_PART out of range"
#endif

}  // namespace permk
