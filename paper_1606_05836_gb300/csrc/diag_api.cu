// Diagnostics of the C ABI: the FP64 FMA throughput probe that sets the peak the
// permanent kernels are measured against.
#include <cuda_runtime.h>
#include <stdint.h>

#include "host_util.h"
#include "perm.h"

namespace {

// Every thread runs PERM_FP64_PROBE_CHAINS independent chains x <- x * a + b for
// `iters` steps: one DFMA per chain and step.  The result is stored only if it
// equals `never` (a value the caller chooses so that the store does not happen),
// so the chains stay live without a store per thread.
__global__ void fp64_fma_probe_kernel(double a, double b, double never, int iters, double* sink) {
  double x[PERM_FP64_PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PERM_FP64_PROBE_CHAINS; c++) x[c] = (double)(threadIdx.x + c) * 1e-3;
#pragma unroll 4
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int c = 0; c < PERM_FP64_PROBE_CHAINS; c++) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < PERM_FP64_PROBE_CHAINS; c++) s += x[c];
  if (s == never) sink[0] = s;
}

}  // namespace

extern "C" int perm_fp64_fma_probe(int iters, int grid, int block, double* dSink, void* stream) {
  permk::NvtxRange nvtx_range("perm_fp64_fma_probe");
  if (iters < 1 || grid < 1 || block < 32 || block > 1024 || (block & 31) || !dSink) return PERM_EINVAL;
  // a < 1 keeps the chains bounded (they converge to b / (1 - a)); the sink value
  // is never reached.
  fp64_fma_probe_kernel<<<grid, block, 0, (cudaStream_t)stream>>>(0.999999, 1e-6, -1.0, iters, dSink);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    permk::record_cuda_error((int)e);
    return PERM_ECUDA;
  }
  return PERM_OK;
}
