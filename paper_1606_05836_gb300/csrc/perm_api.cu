// C ABI of libperm: argument checks, launch planning and dispatch to the
// templated kernels.  The declarations and their contracts are in include/perm.h.
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>
#include <stdlib.h>

#include <mutex>

#include "fwd_kernel.cuh"
#include "host_util.h"
#include "perm.h"

using permk::dd;

namespace {

thread_local int g_last_cuda = 0;

int fail_cuda(cudaError_t e) {
  g_last_cuda = (int)e;
  return PERM_ECUDA;
}

int fail_cuda_int(int e) {
  g_last_cuda = e;
  return PERM_ECUDA;
}

// Instruction-mix override for tuning runs (PERM_TUNE=0..3); -1 = library default.
int tune_override() {
  static int cached = -2;
  if (cached == -2) {
    const char* s = getenv("PERM_TUNE");
    cached = (s && *s) ? atoi(s) : -1;
  }
  return cached;
}

int dispatch_launch(int n, const permk::FwdArgs& a, int prec, int tune, int grid, int block, cudaStream_t s) {
  switch (n) {
#define PERM_CASE(N) \
  case N:            \
    return permk::launch_fwd<N>(a, prec, tune, grid, block, s);
    PERM_CASE(1) PERM_CASE(2) PERM_CASE(3) PERM_CASE(4) PERM_CASE(5) PERM_CASE(6) PERM_CASE(7) PERM_CASE(8)
    PERM_CASE(9) PERM_CASE(10) PERM_CASE(11) PERM_CASE(12) PERM_CASE(13) PERM_CASE(14) PERM_CASE(15)
    PERM_CASE(16) PERM_CASE(17) PERM_CASE(18) PERM_CASE(19) PERM_CASE(20) PERM_CASE(21) PERM_CASE(22)
    PERM_CASE(23) PERM_CASE(24) PERM_CASE(25) PERM_CASE(26) PERM_CASE(27) PERM_CASE(28) PERM_CASE(29)
    PERM_CASE(30) PERM_CASE(31) PERM_CASE(32) PERM_CASE(33) PERM_CASE(34) PERM_CASE(35) PERM_CASE(36)
    PERM_CASE(37) PERM_CASE(38) PERM_CASE(39) PERM_CASE(40) PERM_CASE(41) PERM_CASE(42) PERM_CASE(43)
    PERM_CASE(44) PERM_CASE(45) PERM_CASE(46) PERM_CASE(47) PERM_CASE(48)
#undef PERM_CASE
    default:
      return (int)cudaErrorInvalidValue;
  }
}

int dispatch_occupancy(int n, int prec, int tune, int block, int kind, int* out) {
  switch (n) {
#define PERM_CASE(N) \
  case N:            \
    return permk::fwd_blocks_per_sm<N>(prec, tune, block, kind, out);
    PERM_CASE(1) PERM_CASE(2) PERM_CASE(3) PERM_CASE(4) PERM_CASE(5) PERM_CASE(6) PERM_CASE(7) PERM_CASE(8)
    PERM_CASE(9) PERM_CASE(10) PERM_CASE(11) PERM_CASE(12) PERM_CASE(13) PERM_CASE(14) PERM_CASE(15)
    PERM_CASE(16) PERM_CASE(17) PERM_CASE(18) PERM_CASE(19) PERM_CASE(20) PERM_CASE(21) PERM_CASE(22)
    PERM_CASE(23) PERM_CASE(24) PERM_CASE(25) PERM_CASE(26) PERM_CASE(27) PERM_CASE(28) PERM_CASE(29)
    PERM_CASE(30) PERM_CASE(31) PERM_CASE(32) PERM_CASE(33) PERM_CASE(34) PERM_CASE(35) PERM_CASE(36)
    PERM_CASE(37) PERM_CASE(38) PERM_CASE(39) PERM_CASE(40) PERM_CASE(41) PERM_CASE(42) PERM_CASE(43)
    PERM_CASE(44) PERM_CASE(45) PERM_CASE(46) PERM_CASE(47) PERM_CASE(48)
#undef PERM_CASE
    default:
      return (int)cudaErrorInvalidValue;
  }
}

struct Plan {
  int prec, tune, chunk_log2, block, grid;
  uint64_t per_q, per_r;
};

int sm_count(int* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_cuda(e);
  e = cudaDeviceGetAttribute(out, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail_cuda(e);
  return PERM_OK;
}

int read_opts(const perm_opts* o, int* prec, int* chunk_log2, int* block, int* grid) {
  *prec = o ? o->prec : PERM_FP64;
  // R4 re-splits its double-float row sums from exact FP64 sums more often
  *chunk_log2 = (o && o->chunk_log2) ? o->chunk_log2 : ((o && o->prec == PERM_FP32X2) ? 10 : 12);
  *block = (o && o->block) ? o->block : 128;
  *grid = o ? o->grid : 0;
  if (*prec < PERM_FP64 || *prec > PERM_FP32X2) return PERM_EINVAL;
  if (*chunk_log2 < 1 || *chunk_log2 > 30) return PERM_EINVAL;
  if (*block < 32 || *block > 256 || (*block & 31)) return PERM_EINVAL;
  if (*grid < 0) return PERM_EINVAL;
  return PERM_OK;
}

// Full grid for a kernel instance: SMs x resident blocks per SM, so that every
// SM sub-partition holds the same number of warps (one wave, equal work).
int full_grid(int n, int kind, int prec, int tune, int block, int* grid) {
  int sms = 0, bps = 0;
  int st = sm_count(&sms);
  if (st) return st;
  int e = dispatch_occupancy(n, prec, tune, block, kind, &bps);
  if (e) return fail_cuda_int(e);
  if (bps < 1) return fail_cuda(cudaErrorInvalidConfiguration);
  *grid = sms * bps;
  return PERM_OK;
}

int plan_fwd(int n, int kind, uint64_t range, const perm_opts* o, Plan* p) {
  int grid_opt = 0;
  int st = read_opts(o, &p->prec, &p->chunk_log2, &p->block, &grid_opt);
  if (st) return st;
  if (p->prec == PERM_FP32X2 && kind != permk::KIND_GLYNN) return PERM_EINVAL;  // R4 is a Glynn walk
  p->tune = tune_override();
  if (grid_opt > 0) {
    p->grid = grid_opt;
  } else {
    // At most two resident blocks per SM (two warps per SM sub-partition keep the
    // FP64 pipe busy; a third only adds chunk-start recomputation and staging:
    // measured 2-7 % slower at n = 22-26), and one per SM while a thread would
    // get fewer than 64 Gray indices (n = 20 Glynn: 156 us instead of 211 us).
    int sms = 0, bps = 0;
    st = sm_count(&sms);
    if (st) return st;
    int e = dispatch_occupancy(n, p->prec, p->tune, p->block, kind, &bps);
    if (e) return fail_cuda_int(e);
    if (bps < 1) return fail_cuda(cudaErrorInvalidConfiguration);
    if (bps > 2) bps = 2;
    if (range < (uint64_t)sms * (uint64_t)p->block * 64ull) bps = 1;
    const int g = sms * bps;
    const uint64_t need = (range + (uint64_t)p->block - 1) / (uint64_t)p->block;
    p->grid = (uint64_t)g < need ? g : (int)(need > 0 ? need : 1);
  }
  const uint64_t P = (uint64_t)p->grid * (uint64_t)p->block;
  p->per_q = range / P;
  p->per_r = range % P;
  return PERM_OK;
}

// (sh, sl) += (h, l) in double-double: Knuth's TwoSum of the high parts, the
// low parts added to its error, then renormalised.
void host_dd_add(double& sh, double& sl, double h, double l) {
  const double s = sh + h;
  const double bv = s - sh;
  double e = (sh - (s - bv)) + (h - bv);
  e += sl + l;
  sh = s + e;
  sl = e - (sh - s);
}

size_t workspace_for_grid(int grid) { return 256 + (size_t)grid * 4 * sizeof(double); }

__global__ void set_one_kernel(double2* out) { out[0] = make_double2(1.0, 0.0); }

int run_fwd(const perm_c128* dA, int n, int lda, int kind, uint64_t k_begin, uint64_t k_end, int raw,
            perm_c128* dOut, void* dWork, size_t workBytes, const perm_opts* opts, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (n < 0 || n > PERM_MAX_N) return PERM_ERANGE;
  if (!dOut || (n > 0 && !dA)) return PERM_EINVAL;
  if (lda < n) return PERM_EINVAL;
  if (((uintptr_t)dA & 15u) || ((uintptr_t)dOut & 15u)) return PERM_EINVAL;
  if (n == 0) {
    if (raw) return PERM_ERANGE;
    set_one_kernel<<<1, 1, 0, s>>>((double2*)dOut);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PERM_OK : fail_cuda(e);
  }
  const int M = (kind == permk::KIND_RYSER) ? n : n - 1;
  const uint64_t full = 1ull << M;
  if (k_begin > k_end || k_end > full) return PERM_ERANGE;
  Plan p;
  int st = plan_fwd(n, kind, k_end - k_begin, opts, &p);
  if (st) return st;
  if (!dWork || ((uintptr_t)dWork & 15u)) return PERM_EINVAL;
  if (workBytes < workspace_for_grid(p.grid)) return PERM_ENOMEM;
  permk::FwdArgs a;
  a.A = (const double2*)dA;
  a.n = n;
  a.lda = lda;
  a.kind = kind;
  a.chunk_log2 = p.chunk_log2;
  a.k_begin = k_begin;
  a.k_end = k_end;
  a.per_q = p.per_q;
  a.per_r = p.per_r;
  a.neg_zero = -0.0;
  a.ticket = (unsigned*)dWork;
  a.partials = (double*)((char*)dWork + 256);
  a.out = (double2*)dOut;
  a.raw = raw;
  cudaError_t e = cudaMemsetAsync(dWork, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return fail_cuda(e);
  int le = dispatch_launch(n, a, p.prec, p.tune, p.grid, p.block, s);
  if (le) return fail_cuda_int(le);
  return PERM_OK;
}

// --- prob_sample helpers -----------------------------------------------------

struct GatherArgs {
  const double2* U;
  int ldu;
  int n;           // rows of the gathered matrix
  int ncols;       // its columns
  int transpose;   // 0: out[r][c] = U[rows[r]][cols[c]];  1: out[r][c] = U[cols[c]][rows[r]]
  int rows[PERM_MAX_N];
  int cols[PERM_MAX_N];
  double2* out;    // n x ncols, row-major
};

__global__ void gather_ust_kernel(GatherArgs g) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.n * g.ncols; idx += gridDim.x * blockDim.x) {
    const int r = idx / g.ncols, c = idx % g.ncols;
    g.out[idx] = g.transpose ? g.U[(size_t)g.cols[c] * g.ldu + g.rows[r]] : g.U[(size_t)g.rows[r] * g.ldu + g.cols[c]];
  }
}

// Eq. (1): Pr = |Per|^2 * scale, scale = 1 / (prod s_i! prod t_j!)
__global__ void prob_epilogue_kernel(const double2* per, double scale, double* prob) {
  const double2 p = per[0];
  prob[0] = fma(p.x, p.x, p.y * p.y) * scale;
}

size_t prob_ws_offset_res(int n) { return ((size_t)n * n * sizeof(double2) + 255) & ~(size_t)255; }
size_t prob_ws_offset_sub(int n) { return prob_ws_offset_res(n) + 256; }

// --- repeated columns (multiplicity expansion of Eq. (S2)) ---------------------

struct MultPlan {
  int n, g, nfree;
  int fixed;             // group whose first copy has delta = +1
  int role[PERM_MAX_N];  // per group: free column index, -1 fixed singleton, -2 repeated
  int mult[PERM_MAX_N];
  int radix[PERM_MAX_N];
  long long radix_base[PERM_MAX_N];
  long long classes;     // number of classes (combinations of the repeated groups)
  double terms;          // classes x 2^nfree
};

// Groups: c = 0..g-1 with multiplicities m_c (sum n).  A group of m >= 2 copies
// enters through k = the number of its -1 signs (radix m + 1, weight C(m, k));
// singletons are free binary columns.  The delta = +1 copy is taken from a
// singleton if there is one (halving the free range), otherwise from the smallest
// repeated group (its k then runs over 0..m-1 with weight C(m-1, k)).
int mult_plan(int n, int g, const int32_t* mult, MultPlan* P) {
  if (g < 1 || g > n || n > PERM_MAX_N) return PERM_ERANGE;
  int sum = 0;
  for (int c = 0; c < g; c++) {
    if (mult[c] < 1) return PERM_EINVAL;
    sum += mult[c];
    P->mult[c] = mult[c];
  }
  if (sum != n) return PERM_EINVAL;
  P->n = n;
  P->g = g;
  int fixed = -1;
  for (int c = 0; c < g; c++)
    if (mult[c] == 1) {
      fixed = c;
      break;
    }
  if (fixed < 0) {
    fixed = 0;
    for (int c = 1; c < g; c++)
      if (mult[c] < mult[fixed]) fixed = c;
  }
  P->fixed = fixed;
  int nfree = 0;
  long long classes = 1;
  for (int c = 0; c < g; c++) {
    P->radix[c] = 0;
    P->radix_base[c] = 1;
    if (mult[c] == 1) {
      P->role[c] = (c == fixed) ? -1 : nfree++;
    } else {
      P->role[c] = -2;
      P->radix[c] = (c == fixed) ? mult[c] : mult[c] + 1;
      P->radix_base[c] = classes;
      classes *= P->radix[c];  // <= 2^(n-1) <= 2^47: a group of m copies has m + 1 <= 2^m classes
    }
  }
  P->nfree = nfree;
  P->classes = classes;
  P->terms = (double)classes * (double)(1ull << nfree);
  return PERM_OK;
}

int run_mult(const perm_c128* dB, int n, int ldb, int g, const int32_t* hMult, perm_c128* dOut, void* dWork,
             size_t workBytes, const perm_opts* opts, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!dB || !dOut || !hMult || !dWork) return PERM_EINVAL;
  if (((uintptr_t)dB & 15u) || ((uintptr_t)dOut & 15u) || ((uintptr_t)dWork & 15u)) return PERM_EINVAL;
  if (ldb < g) return PERM_EINVAL;
  MultPlan P;
  int st = mult_plan(n, g, hMult, &P);
  if (st) return st;
  const uint64_t total = (uint64_t)P.classes << P.nfree;
  Plan pl;
  st = plan_fwd(n, permk::KIND_GLYNN_MULT, total, opts, &pl);
  if (st) return st;
  if (workBytes < workspace_for_grid(pl.grid)) return PERM_ENOMEM;
  permk::FwdArgs a;
  a.A = (const double2*)dB;
  a.n = n;
  a.lda = ldb;
  a.kind = permk::KIND_GLYNN_MULT;
  a.chunk_log2 = pl.chunk_log2;
  a.k_begin = 0;
  a.k_end = total;
  a.per_q = pl.per_q;
  a.per_r = pl.per_r;
  a.neg_zero = -0.0;
  a.ticket = (unsigned*)dWork;
  a.partials = (double*)((char*)dWork + 256);
  a.out = (double2*)dOut;
  a.raw = 0;
  a.mult.g = g;
  a.mult.nfree = P.nfree;
  for (int c = 0; c < g; c++) {
    a.mult.role[c] = (signed char)P.role[c];
    a.mult.mult[c] = (unsigned char)P.mult[c];
    a.mult.radix[c] = (unsigned char)P.radix[c];
    a.mult.radix_base[c] = P.radix_base[c];
  }
  cudaError_t e = cudaMemsetAsync(dWork, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return fail_cuda(e);
  int le = dispatch_launch(n, a, pl.prec, pl.tune, pl.grid, pl.block, s);
  if (le) return fail_cuda_int(le);
  return PERM_OK;
}

}  // namespace

void permk::record_cuda_error(int err) { g_last_cuda = err; }

extern "C" {

size_t perm_workspace_size(int n, const perm_opts* opts) {
  if (n < 1 || n > PERM_MAX_N) return workspace_for_grid(1);
  int prec, chunk, block, grid_opt;
  if (read_opts(opts, &prec, &chunk, &block, &grid_opt)) return 0;
  if (grid_opt > 0) return workspace_for_grid(grid_opt);
  int g0 = 0, g1 = 0;
  if (full_grid(n, permk::KIND_GLYNN, prec, tune_override(), block, &g0)) return 0;
  if (full_grid(n, permk::KIND_RYSER, prec, tune_override(), block, &g1)) return 0;
  return workspace_for_grid(g0 > g1 ? g0 : g1);
}

int perm_glynn(const perm_c128* dA, int n, int lda, perm_c128* dOut, void* dWork, size_t workBytes,
               const perm_opts* opts, void* stream) {
  permk::NvtxRange nvtx_range("perm_glynn");
  const uint64_t full = (n >= 1 && n <= PERM_MAX_N) ? (1ull << (n - 1)) : 0;
  return run_fwd(dA, n, lda, permk::KIND_GLYNN, 0, full, 0, dOut, dWork, workBytes, opts, stream);
}

int perm_ryser(const perm_c128* dA, int n, int lda, perm_c128* dOut, void* dWork, size_t workBytes,
               const perm_opts* opts, void* stream) {
  permk::NvtxRange nvtx_range("perm_ryser");
  const uint64_t full = (n >= 1 && n <= PERM_MAX_N) ? (1ull << n) : 0;
  return run_fwd(dA, n, lda, permk::KIND_RYSER, 0, full, 0, dOut, dWork, workBytes, opts, stream);
}

int perm_ryser_nw(const perm_c128* dA, int n, int lda, perm_c128* dOut, void* dWork, size_t workBytes,
                  const perm_opts* opts, void* stream) {
  permk::NvtxRange nvtx_range("perm_ryser_nw");
  const uint64_t full = (n >= 1 && n <= PERM_MAX_N) ? (1ull << (n - 1)) : 0;
  return run_fwd(dA, n, lda, permk::KIND_RYSER_NW, 0, full, 0, dOut, dWork, workBytes, opts, stream);
}

int perm_glynn_range(const perm_c128* dA, int n, int lda, uint64_t k_begin, uint64_t k_end, perm_c128* dOut,
                     void* dWork, size_t workBytes, const perm_opts* opts, void* stream) {
  permk::NvtxRange nvtx_range("perm_glynn_range");
  if (n < 1) return PERM_ERANGE;
  return run_fwd(dA, n, lda, permk::KIND_GLYNN, k_begin, k_end, 1, dOut, dWork, workBytes, opts, stream);
}

int perm_ryser_range(const perm_c128* dA, int n, int lda, uint64_t k_begin, uint64_t k_end, perm_c128* dOut,
                     void* dWork, size_t workBytes, const perm_opts* opts, void* stream) {
  permk::NvtxRange nvtx_range("perm_ryser_range");
  if (n < 1) return PERM_ERANGE;
  return run_fwd(dA, n, lda, permk::KIND_RYSER, k_begin, k_end, 1, dOut, dWork, workBytes, opts, stream);
}


int perm_combine_partials(const perm_c128* hParts, int count, int n, int method, perm_c128* hOut) {
  if (!hParts || !hOut || count < 1 || (method != 0 && method != 1)) return PERM_EINVAL;
  if (n < 1 || n > PERM_MAX_N) return PERM_ERANGE;
  // double-double sum in the given order (TwoSum of the high parts, low parts
  // added, renormalised), then the exact scaling of the formula
  double rh = 0.0, rl = 0.0, ih = 0.0, il = 0.0;
  for (int p = 0; p < count; p++) {
    const perm_c128 hi = hParts[2 * p], lo = hParts[2 * p + 1];
    host_dd_add(rh, rl, hi.re, lo.re);
    host_dd_add(ih, il, hi.im, lo.im);
  }
  double f = 1.0;
  int e = 0;
  if (method == 0) e = -(n - 1);
  else if (n & 1) f = -1.0;
  hOut[0].re = ldexp(rh, e) * f;
  hOut[0].im = ldexp(ih, e) * f;
  hOut[1].re = ldexp(rl, e) * f;
  hOut[1].im = ldexp(il, e) * f;
  return PERM_OK;
}

size_t perm_glynn_mult_workspace_size(int n, int g, const int32_t* hMult, const perm_opts* opts) {
  if (!hMult || n < 1) return 0;
  MultPlan P;
  if (mult_plan(n, g, hMult, &P)) return 0;
  return perm_workspace_size(n, opts);
}

int perm_glynn_mult(const perm_c128* dB, int n, int ldb, int g, const int32_t* hMult, perm_c128* dOut, void* dWork,
                    size_t workBytes, const perm_opts* opts, void* stream) {
  permk::NvtxRange nvtx_range("perm_glynn_mult");
  if (n < 1 || n > PERM_MAX_N) return PERM_ERANGE;
  return run_mult(dB, n, ldb, g, hMult, dOut, dWork, workBytes, opts, stream);
}

size_t prob_sample_workspace_size(int n, const perm_opts* opts) {
  if (n < 0 || n > PERM_MAX_N) return 0;
  const size_t fwd = n >= 1 ? perm_workspace_size(n, opts) : 256;
  if (fwd == 0) return 0;
  return prob_ws_offset_sub(n) + fwd;  // gathered matrix + result + kernel workspace
}

int prob_sample(const perm_c128* dU, int m, int ldu, const int32_t* hS, const int32_t* hT, double* hProb,
                perm_c128* hPerm, void* dWork, size_t workBytes, const perm_opts* opts, void* stream) {
  permk::NvtxRange nvtx_range("prob_sample");
  cudaStream_t s = (cudaStream_t)stream;
  if (m < 1 || !dU || ldu < m || !hS || !hT || !hProb || !dWork) return PERM_EINVAL;
  if (((uintptr_t)dU & 15u) || ((uintptr_t)dWork & 255u)) return PERM_EINVAL;
  int rows[PERM_MAX_N], cols[PERM_MAX_N];           // input / output mode of every row / column of U_ST
  int ins[PERM_MAX_N], s_mult[PERM_MAX_N], outs[PERM_MAX_N], t_mult[PERM_MAX_N];
  int n = 0, nt = 0, gi = 0, go = 0;
  bool rep_s = false, rep_t = false;
  double denom = 1.0;
  for (int i = 0; i < m; i++) {
    if (hS[i] < 0 || hT[i] < 0) return PERM_EINVAL;
    if (hS[i] > PERM_MAX_N || hT[i] > PERM_MAX_N) return PERM_ERANGE;
    for (int k = 2; k <= hS[i]; k++) denom *= (double)k;
    for (int k = 2; k <= hT[i]; k++) denom *= (double)k;
    if (hS[i] > 0) {
      if (gi >= PERM_MAX_N) return PERM_ERANGE;
      ins[gi] = i;
      s_mult[gi++] = hS[i];
      rep_s = rep_s || hS[i] > 1;
    }
    if (hT[i] > 0) {
      if (go >= PERM_MAX_N) return PERM_ERANGE;
      outs[go] = i;
      t_mult[go++] = hT[i];
      rep_t = rep_t || hT[i] > 1;
    }
    for (int k = 0; k < hS[i]; k++) {
      if (n >= PERM_MAX_N) return PERM_ERANGE;
      rows[n++] = i;
    }
    for (int k = 0; k < hT[i]; k++) {
      if (nt >= PERM_MAX_N) return PERM_ERANGE;
      cols[nt++] = i;
    }
  }
  if (n != nt) return PERM_EINVAL;
  if (workBytes < prob_sample_workspace_size(n, opts)) return PERM_ENOMEM;
  char* w = (char*)dWork;
  double2* mat = (double2*)w;
  double2* res = (double2*)(w + prob_ws_offset_res(n));
  double* prob = (double*)(w + prob_ws_offset_res(n) + 64);
  char* sub = w + prob_ws_offset_sub(n);
  const size_t sub_bytes = workBytes - prob_ws_offset_sub(n);
  GatherArgs g;
  g.U = (const double2*)dU;
  g.ldu = ldu;
  g.n = n;
  g.out = mat;
  int st = PERM_OK;
  // Photon collisions: repeated columns of U_ST (an output mode with t_j > 1) or
  // repeated rows (s_i > 1, handled as columns of the transpose) go through the
  // multiplicity expansion; the orientation with fewer terms is used.
  int orient = 0;  // 0: plain; 1: columns = distinct outputs; 2: columns = distinct inputs
  if (n > 0 && (rep_s || rep_t)) {
    MultPlan pc, pr;
    const bool ok_c = mult_plan(n, go, t_mult, &pc) == PERM_OK;
    const bool ok_r = mult_plan(n, gi, s_mult, &pr) == PERM_OK;
    if (ok_c && (!ok_r || pc.terms <= pr.terms)) orient = 1;
    else if (ok_r) orient = 2;
  }
  if (orient == 1) {
    for (int r = 0; r < n; r++) g.rows[r] = rows[r];
    for (int c = 0; c < go; c++) g.cols[c] = outs[c];
    g.ncols = go;
    g.transpose = 0;
  } else if (orient == 2) {
    for (int r = 0; r < n; r++) g.rows[r] = cols[r];
    for (int c = 0; c < gi; c++) g.cols[c] = ins[c];
    g.ncols = gi;
    g.transpose = 1;
  } else {
    for (int r = 0; r < n; r++) {
      g.rows[r] = rows[r];
      g.cols[r] = cols[r];
    }
    g.ncols = n;
    g.transpose = 0;
  }
  if (n > 0) {
    gather_ust_kernel<<<(n * g.ncols + 255) / 256, 256, 0, s>>>(g);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(e);
  }
  if (orient == 1) {
    st = run_mult((const perm_c128*)mat, n, go, go, t_mult, (perm_c128*)res, sub, sub_bytes, opts, stream);
  } else if (orient == 2) {
    st = run_mult((const perm_c128*)mat, n, gi, gi, s_mult, (perm_c128*)res, sub, sub_bytes, opts, stream);
  } else {
    st = run_fwd((const perm_c128*)mat, n, n, permk::KIND_GLYNN, 0, n >= 1 ? (1ull << (n - 1)) : 0, 0,
                 (perm_c128*)res, sub, sub_bytes, opts, stream);
  }
  if (st) return st;
  prob_epilogue_kernel<<<1, 1, 0, s>>>(res, 1.0 / denom, prob);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_cuda(e);
  e = cudaMemcpyAsync(hProb, prob, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return fail_cuda(e);
  if (hPerm) {
    e = cudaMemcpyAsync(hPerm, res, sizeof(perm_c128), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return fail_cuda(e);
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_cuda(e);
  return PERM_OK;
}

const char* perm_strerror(int status) {
  switch (status) {
    case PERM_OK: return "ok";
    case PERM_EINVAL: return "invalid argument";
    case PERM_ERANGE: return "size or index range out of bounds";
    case PERM_ENOMEM: return "workspace too small";
    case PERM_ECUDA: return "CUDA runtime error";
    case PERM_ENONFINITE: return "non-finite value";
    case PERM_ETIMEOUT: return "bounded wait timed out";
    default: return "unknown status";
  }
}

int perm_last_cuda_error(void) { return g_last_cuda; }

int perm_version(void) { return PERM_ABI_VERSION; }

}  // extern "C"

// ---------------------------------------------------------------------------
// perm_glynn_noalloc: the Glynn kernel with its scratch in a fixed device array
// ---------------------------------------------------------------------------
//
// Scratch of the single-permanent kernel = a 256-byte header (the last-block
// ticket) + 32 bytes of double-double partial sums per block.  Here it lives in
// one file-scope device array instead of a caller workspace, for callers that
// may not allocate device memory themselves.  Every GPU that loads this library
// holds the array (PERM_NOALLOC_SCRATCH_BYTES) until the process exits.

static __device__ __align__(256) unsigned char g_noalloc_scratch[PERM_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached.
int noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_cuda(e);
  if (dev < 0 || dev >= kMaxDevices) return PERM_EINVAL;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return fail_cuda(e);
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  return PERM_OK;
}

}  // namespace

extern "C" int perm_glynn_noalloc(const perm_c128* dA, int n, int lda, perm_c128* dOut, const perm_opts* opts,
                                  void* stream) {
  permk::NvtxRange nvtx_range("perm_glynn_noalloc");
  if (n < 0 || n > PERM_MAX_N) return PERM_ERANGE;
  if (!dOut || (n > 0 && !dA)) return PERM_EINVAL;
  void* scratch = nullptr;
  int st = noalloc_scratch(&scratch);
  if (st) return st;
  if (n >= 1) {
    // the launch this call would make must fit the fixed partial-sum array
    Plan p;
    st = plan_fwd(n, permk::KIND_GLYNN, 1ull << (n - 1), opts, &p);
    if (st) return st;
    if (workspace_for_grid(p.grid) > (size_t)PERM_NOALLOC_SCRATCH_BYTES) return PERM_ENOMEM;
  }
  // run_fwd zeroes the ticket (the only scratch that must start at zero) with
  // cudaMemsetAsync before the launch; partials are written before they are read.
  const uint64_t full = (n >= 1) ? (1ull << (n - 1)) : 0;
  return run_fwd(dA, n, lda, permk::KIND_GLYNN, 0, full, 0, dOut, scratch, (size_t)PERM_NOALLOC_SCRATCH_BYTES, opts,
                 stream);
}
