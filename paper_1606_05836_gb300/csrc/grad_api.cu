// C ABI of the adjoint: perm_grad_workspace_size / perm_grad (declared in perm.h).
#include <cuda_runtime.h>
#include <stdint.h>

#include "grad_kernel.cuh"
#include "host_util.h"
#include "perm.h"

namespace permk {

// One block per (i, j): sum of G_ij over the lane pairs in a fixed order.
__global__ void __launch_bounds__(256) grad_reduce_kernel(GradReduceArgs r) {
  const int n = r.n;
  const int ij = blockIdx.x;
  const int i = ij / n, j = ij % n;
  __shared__ dd red[2][8];
  const double2* base = r.state + (long long)(i * n + j) * r.P;
  dd tr{0.0, 0.0}, ti{0.0, 0.0};
  for (long long T = threadIdx.x; T < r.P; T += blockDim.x) {
    const double2 v = base[T];
    tr = dd_add(tr, dd{v.x, 0.0});
    ti = dd_add(ti, dd{v.y, 0.0});
  }
  warp_sum_dd(tr, ti);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[0][warp] = tr;
    red[1][warp] = ti;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    tr = red[0][0];
    ti = red[1][0];
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
      tr = dd_add(tr, red[0][w]);
      ti = dd_add(ti, red[1][w]);
    }
    // forward permanent from the block partials of the walk kernel
    dd pr{0.0, 0.0}, pi{0.0, 0.0};
    for (int blk = 0; blk < r.nblocks; blk++) {
      pr = dd_add(pr, dd{r.partials[4 * blk], r.partials[4 * blk + 1]});
      pi = dd_add(pi, dd{r.partials[4 * blk + 2], r.partials[4 * blk + 3]});
    }
    // both lanes of every pair added each term: one more factor 1/2
    const int sum_s = r.scale_exp[0];
    const double Pre = ldexp(pr.hi + pr.lo, -sum_s - (n - 1) - 1);
    const double Pim = ldexp(pi.hi + pi.lo, -sum_s - (n - 1) - 1);
    // rows were scaled by 2^{s_i}: dPer/da_ij = 2^{s_i - sum s - (n-1)} G'_ij
    const int e = r.scale_exp[1 + i] - sum_s - (n - 1);
    const double mr = ldexp(tr.hi + tr.lo, e);
    const double mi = ldexp(ti.hi + ti.lo, e);
    if (r.minor) r.minor[ij] = make_double2(mr, mi);
    if (r.grad_abs2) {
      // 2 Per conj(M): d|Per|^2/dRe a + i d|Per|^2/dIm a
      r.grad_abs2[ij] = make_double2(2.0 * (Pre * mr + Pim * mi), 2.0 * (Pim * mr - Pre * mi));
    }
    if (ij == 0) {
      if (r.perm) r.perm[0] = make_double2(Pre, Pim);
      if (r.abs2) r.abs2[0] = fma(Pre, Pre, Pim * Pim);
    }
  }
}

}  // namespace permk

namespace {

using namespace permk;

int gfail(int e) {
  record_cuda_error(e);
  return PERM_ECUDA;
}

#define PERM_G_CASES(X)                                                                                   \
  X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) X(17) X(18) X(19) \
  X(20) X(21) X(22) X(23) X(24) X(25) X(26) X(27) X(28) X(29) X(30) X(31) X(32)

int dispatch_grad(int n, const GradArgs& a, int prec, int grid, cudaStream_t s) {
  switch (n) {
#define PERM_GC(N) \
  case N:          \
    return launch_grad<N>(a, prec, grid, s);
    PERM_G_CASES(PERM_GC)
#undef PERM_GC
    default:
      return (int)cudaErrorInvalidValue;
  }
}

int dispatch_grad_occupancy(int n, int prec, int* out) {
  switch (n) {
#define PERM_GC(N) \
  case N:          \
    return grad_blocks_per_sm<N>(prec, out);
    PERM_G_CASES(PERM_GC)
#undef PERM_GC
    default:
      return (int)cudaErrorInvalidValue;
  }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct GradLayout {
  int grid, chunk_log2, prec;
  long long P;
  size_t scale_exp, partials, state, total;
};

int grad_layout(int n, const perm_opts* o, GradLayout* L) {
  if (n < 1 || n > PERM_GRAD_MAX_N) return PERM_ERANGE;
  L->prec = o ? o->prec : PERM_FP64;
  if (L->prec != PERM_FP64 && L->prec != PERM_FP64_DF) return PERM_EINVAL;
  if (o && o->block != 0 && o->block != GRAD_BLOCK) return PERM_EINVAL;
  L->chunk_log2 = (o && o->chunk_log2) ? o->chunk_log2 : 12;
  if (L->chunk_log2 < 1 || L->chunk_log2 > 30) return PERM_EINVAL;
  int grid = o ? o->grid : 0;
  if (grid < 0) return PERM_EINVAL;
  if (grid == 0) {
    int dev = 0, sms = 0, bps = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return gfail((int)e);
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return gfail((int)e);
    int oe = dispatch_grad_occupancy(n, L->prec, &bps);
    if (oe) return gfail(oe);
    if (bps < 1) return gfail((int)cudaErrorInvalidConfiguration);
    grid = sms * bps;
  }
  L->grid = grid;
  L->P = (long long)grid * (GRAD_BLOCK / 2);  // lane pairs
  size_t off = 0;
  L->scale_exp = off;
  off = align256(off + sizeof(int) * (size_t)(1 + n));
  L->partials = off;
  off = align256(off + 32 * (size_t)grid);
  L->state = off;
  off = align256(off + sizeof(double2) * (size_t)n * n * (size_t)L->P);
  L->total = off;
  return PERM_OK;
}

__global__ void grad_trivial_kernel(double2* perm, double* abs2, int batch) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  if (perm) perm[b] = make_double2(1.0, 0.0);
  if (abs2) abs2[b] = 1.0;
}

}  // namespace

extern "C" {

size_t perm_grad_workspace_size(int n, const perm_opts* opts) {
  if (n == 0) return 256;
  GradLayout L;
  if (grad_layout(n, opts, &L)) return 0;
  return L.total;
}

int perm_grad(const perm_c128* dA, int n, int lda, int batch, int64_t strideA, perm_c128* dPerm, double* dAbs2,
              perm_c128* dMinor, perm_c128* dGradAbs2, void* dWork, size_t workBytes, const perm_opts* opts,
              void* stream) {
  permk::NvtxRange nvtx_range("perm_grad");
  cudaStream_t s = (cudaStream_t)stream;
  if (n < 0 || n > PERM_GRAD_MAX_N) return PERM_ERANGE;
  if (batch < 0) return PERM_EINVAL;
  if (batch == 0) return PERM_OK;
  if (!dPerm && !dAbs2 && !dMinor && !dGradAbs2) return PERM_EINVAL;
  if (n > 0 && (!dA || lda < n || strideA < (int64_t)(n - 1) * lda + n)) return PERM_EINVAL;
  if (((uintptr_t)dA & 15u) || ((uintptr_t)dPerm & 15u) || ((uintptr_t)dMinor & 15u) ||
      ((uintptr_t)dGradAbs2 & 15u))
    return PERM_EINVAL;
  if (n == 0) {
    grad_trivial_kernel<<<(batch + 127) / 128, 128, 0, s>>>((double2*)dPerm, dAbs2, batch);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PERM_OK : gfail((int)e);
  }
  GradLayout L;
  int st = grad_layout(n, opts, &L);
  if (st) return st;
  if (!dWork || ((uintptr_t)dWork & 255u)) return PERM_EINVAL;
  if (workBytes < L.total) return PERM_ENOMEM;
  char* w = (char*)dWork;
  const uint64_t terms = 1ull << (n - 1);
  for (int b = 0; b < batch; b++) {
    GradArgs a;
    a.A = (const double2*)dA + (size_t)b * (size_t)strideA;
    a.lda = lda;
    a.chunk_log2 = L.chunk_log2;
    a.per_q = terms / (uint64_t)L.P;
    a.per_r = terms % (uint64_t)L.P;
    a.neg_zero = -0.0;
    a.state = (double2*)(w + L.state);
    a.P = L.P;
    a.partials = (double*)(w + L.partials);
    a.scale_exp = (int*)(w + L.scale_exp);
    int le = dispatch_grad(n, a, L.prec, L.grid, s);
    if (le) return gfail(le);
    GradReduceArgs r;
    r.state = a.state;
    r.P = L.P;
    r.n = n;
    r.partials = a.partials;
    r.nblocks = L.grid;
    r.scale_exp = a.scale_exp;
    r.perm = dPerm ? (double2*)dPerm + b : nullptr;
    r.abs2 = dAbs2 ? dAbs2 + b : nullptr;
    r.minor = dMinor ? (double2*)dMinor + (size_t)b * n * n : nullptr;
    r.grad_abs2 = dGradAbs2 ? (double2*)dGradAbs2 + (size_t)b * n * n : nullptr;
    grad_reduce_kernel<<<n * n, 256, 0, s>>>(r);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return gfail((int)e);
  }
  return PERM_OK;
}

}  // extern "C"
