// C ABI of the row minors and of the boson-sampling draws (declared in perm.h):
// perm_row_minors_workspace_size / perm_row_minors and
// boson_sample_workspace_size / boson_sample.
//
// A draw follows the chain rule over Eq. (1) of arXiv 1606.05836 (one photon in
// each of n distinct input modes): photons in the caller's random order alpha,
// and for k = 1..n every output mode l is weighted by
//   w_k(l) = |sum_j U[in(alpha_j), l] m_j|^2,  m_j = Per(A[r_<k, cols 0..k-1 without j]),
// A[l, j] = U[in(alpha_j), l]; r_k is the first mode whose running sum of w_k
// exceeds u_k * sum_l w_k(l).  Per step: one minors_kernel<k> launch over all
// draws (the k minors of the (k-1) x k matrix read straight from U), then one
// draw_kernel block per draw (minors from the block partials, weights, running
// sums in mode order by a block scan, choice).  Every launch is stream-ordered; nothing is
// copied to or from the host.
#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>

#include <mutex>

#include "host_util.h"
#include "minors_kernel.cuh"
#include "perm.h"

namespace permk {

struct MinorsReduceArgs {
  const double* partials;  // [item][bpi][k][4]
  int bpi, k;
  const int* scale_exp;    // [item]
  double2* out;            // [item][k]
};

// One block per item; thread j sums column j's block partials in block order.
__global__ void minors_reduce_kernel(MinorsReduceArgs r) {
  const int item = blockIdx.x, j = threadIdx.x;
  if (j >= r.k) return;
  dd tr{0.0, 0.0}, ti{0.0, 0.0};
  for (int blk = 0; blk < r.bpi; blk++) {
    const double* p = r.partials + (((size_t)item * r.bpi + blk) * r.k + j) * 4;
    tr = dd_add(tr, dd{p[0], p[1]});
    ti = dd_add(ti, dd{p[2], p[3]});
  }
  // rows were scaled by 2^{s_i}; Glynn's normalisation is 2^-(k-1)
  const int e = -r.scale_exp[item] - (r.k - 1);
  r.out[(size_t)item * r.k + j] = make_double2(ldexp(tr.hi + tr.lo, e), ldexp(ti.hi + ti.lo, e));
}

__global__ void minors_one_kernel(double2* out, int batch) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < batch) out[b] = make_double2(1.0, 0.0);
}

constexpr int SAMPLE_MAX_N = 32;

struct SampleInitArgs {
  int n, nsamples;
  int inputs[SAMPLE_MAX_N];
  const int* alpha;     // [s][n]
  const double* unif;   // [s][n]
  int* cmap;            // [s][n] input mode of photon column j
  int* status;          // [s]: 0 ok, 1 a step had no positive weight, 2 invalid draw inputs
  int* R;               // [s][n]
};

// Checks each draw's alpha (a permutation of 0..n-1) and u (in [0, 1)), maps the
// photon columns to input modes and marks every output slot -1.
__global__ void sample_init_kernel(SampleInitArgs a) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.nsamples) return;
  const int n = a.n;
  unsigned long long seen = 0ull;
  bool ok = true;
  for (int j = 0; j < n; j++) {
    const int aj = a.alpha[s * n + j];
    if (aj < 0 || aj >= n || ((seen >> aj) & 1ull)) ok = false;
    else seen |= 1ull << aj;
    const double u = a.unif[s * n + j];
    if (!(u >= 0.0 && u < 1.0)) ok = false;
  }
  for (int j = 0; j < n; j++) {
    a.cmap[s * n + j] = ok ? a.inputs[a.alpha[s * n + j]] : 0;
    a.R[s * n + j] = -1;
  }
  a.status[s] = ok ? 0 : 2;
}

struct DrawArgs {
  const double2* U;
  long long ldu;
  int m, n, k;          // step k = 1..n
  const int* cmap;
  const double* unif;
  int* R;
  int* status;
  const double* partials;  // [s][bpi][k][4] (unused at k = 1)
  int bpi;
  double* w;            // [s][m] weights
  double* cum;          // [s][m] running sums
};

constexpr int DRAW_BLOCK = 512;
constexpr int DRAW_TILE = 2 * DRAW_BLOCK;

__global__ void __launch_bounds__(DRAW_BLOCK) draw_kernel(DrawArgs a) {
  const long long s = blockIdx.x;
  const int k = a.k, n = a.n, m = a.m;
  __shared__ double2 mnr[SAMPLE_MAX_N];
  __shared__ int s_cm[SAMPLE_MAX_N];
  __shared__ double s_W;
  __shared__ int s_first, s_last;
  if (a.status[s] != 0) return;  // failed or invalid: its slots already hold -1
  if (threadIdx.x < k) {
    const int j = threadIdx.x;
    s_cm[j] = a.cmap[s * n + j];
    if (k == 1) {
      mnr[0] = make_double2(1.0, 0.0);
    } else {
      // the minors up to the common factor 2^{-(k-1) - sum s_i}, which cancels in w / W
      dd tr{0.0, 0.0}, ti{0.0, 0.0};
      for (int blk = 0; blk < a.bpi; blk++) {
        const double* p = a.partials + (((size_t)s * a.bpi + blk) * k + j) * 4;
        tr = dd_add(tr, dd{p[0], p[1]});
        ti = dd_add(ti, dd{p[2], p[3]});
      }
      mnr[j] = make_double2(tr.hi + tr.lo, ti.hi + ti.lo);
    }
  }
  if (threadIdx.x == 0) {
    s_first = INT_MAX;
    s_last = -1;
  }
  __syncthreads();
  double* w = a.w + s * m;
  double* cum = a.cum + s * m;
  // Tiles of DRAW_TILE modes (two per thread): the block computes
  // w(l) = |sum_j A[l, j] m_j|^2, A[l, j] = U[in(alpha_j), l] (coalesced over l),
  // then the running sums of the tile by a block-wide scan in a fixed order
  // (thread pair sums, warp shuffles, warp totals), carried across tiles.
  __shared__ double wt[DRAW_TILE], ct[DRAW_TILE];
  __shared__ double wsum[DRAW_BLOCK / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double carry = 0.0;  // the same value in every thread
  for (int l0 = 0; l0 < m; l0 += DRAW_TILE) {
    const int len = (m - l0 < DRAW_TILE) ? m - l0 : DRAW_TILE;
    for (int t = threadIdx.x; t < DRAW_TILE; t += blockDim.x) {
      double wv = 0.0;
      if (t < len) {
        const int l = l0 + t;
        double ar = 0.0, ai = 0.0;
#pragma unroll 8
        for (int j = 0; j < k; j++) {
          const double2 u = a.U[(long long)s_cm[j] * a.ldu + l];
          const double2 mm = mnr[j];
          ar = fma(u.x, mm.x, ar);
          ar = fma(-u.y, mm.y, ar);
          ai = fma(u.x, mm.y, ai);
          ai = fma(u.y, mm.x, ai);
        }
        wv = fma(ar, ar, ai * ai);
      }
      wt[t] = wv;
    }
    __syncthreads();
    const double a0 = wt[2 * threadIdx.x], a1 = wt[2 * threadIdx.x + 1];
    const double pair = a0 + a1;
    double inc = pair;  // inclusive scan of the pair sums within the warp
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const double o = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += o;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      double v = lane < DRAW_BLOCK / 32 ? wsum[lane] : 0.0;
#pragma unroll
      for (int off = 1; off < DRAW_BLOCK / 32; off <<= 1) {
        const double o = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += o;
      }
      if (lane < DRAW_BLOCK / 32) wsum[lane] = v;  // inclusive warp prefixes
    }
    __syncthreads();
    const double before = carry + ((warp > 0 ? wsum[warp - 1] : 0.0) + (inc - pair));
    ct[2 * threadIdx.x] = before + a0;
    ct[2 * threadIdx.x + 1] = (before + a0) + a1;
    carry = carry + wsum[DRAW_BLOCK / 32 - 1];
    __syncthreads();
    for (int t = threadIdx.x; t < len; t += blockDim.x) {
      w[l0 + t] = wt[t];
      cum[l0 + t] = ct[t];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) s_W = carry;
  __syncthreads();
  const double W = s_W;
  if (!(W > 0.0) || !isfinite(W)) {
    // no mode can be drawn: the draw fails (all its slots -1)
    for (int j = threadIdx.x; j < n; j += blockDim.x) a.R[s * n + j] = -1;
    if (threadIdx.x == 0) a.status[s] = 1;
    return;
  }
  const double x = a.unif[s * n + (k - 1)] * W;
  int first = INT_MAX, last = -1;
  for (int l = threadIdx.x; l < m; l += blockDim.x) {
    if (first == INT_MAX && cum[l] > x) first = l;
    if (w[l] > 0.0) last = l;
  }
  if (first != INT_MAX) atomicMin(&s_first, first);
  if (last >= 0) atomicMax(&s_last, last);
  __syncthreads();
  if (threadIdx.x == 0) {
    // rounding can leave u W at or above every running sum: take the last mode of positive weight
    const int pick = (s_first != INT_MAX) ? s_first : s_last;
    a.R[s * n + (k - 1)] = pick;
  }
}

}  // namespace permk

namespace {

using namespace permk;

int sfail(int e) {
  record_cuda_error(e);
  return PERM_ECUDA;
}

#define PERM_M_CASES(X)                                                                                      \
  X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) X(17) X(18) X(19) X(20) \
  X(21) X(22) X(23) X(24) X(25) X(26) X(27) X(28) X(29) X(30) X(31) X(32)

int dispatch_minors(int k, const MinorsArgs& a, int prec, int grid, cudaStream_t s) {
  switch (k) {
#define PERM_MC(K) \
  case K:          \
    return launch_minors<K>(a, prec, grid, s);
    PERM_M_CASES(PERM_MC)
#undef PERM_MC
    default:
      return (int)cudaErrorInvalidValue;
  }
}

int dispatch_minors_occupancy(int k, int prec, int* out) {
  switch (k) {
#define PERM_MC(K) \
  case K:          \
    return minors_blocks_per_sm<K>(prec, out);
    PERM_M_CASES(PERM_MC)
#undef PERM_MC
    default:
      return (int)cudaErrorInvalidValue;
  }
}

// Resident blocks per SM of minors_kernel<k>, cached per device.
constexpr int MAX_DEVICES = 64;
std::mutex g_occ_mu;
int g_occ[MAX_DEVICES][3][MINORS_MAX_K + 1];
int g_sms[MAX_DEVICES];

int minors_wave(int k, int prec, long long* wave) {
  const int pi = prec == PERM_FP32X2 ? 2 : (prec == PERM_FP64_DF ? 1 : 0);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return sfail((int)e);
  if (dev < 0 || dev >= MAX_DEVICES) return PERM_EINVAL;
  std::lock_guard<std::mutex> lock(g_occ_mu);
  if (g_sms[dev] == 0) {
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return sfail((int)e);
    g_sms[dev] = sms;
  }
  if (g_occ[dev][pi][k] == 0) {
    int bps = 0;
    const int oe = dispatch_minors_occupancy(k, prec, &bps);
    if (oe) return sfail(oe);
    if (bps < 1) return sfail((int)cudaErrorInvalidConfiguration);
    g_occ[dev][pi][k] = bps;
  }
  *wave = (long long)g_sms[dev] * g_occ[dev][pi][k];
  return PERM_OK;
}

struct MinorsPlan {
  int bpi, chunk_log2, prec;
  uint64_t per_q, per_r;
};

// FP64 (R0), R3 or R4; R4's default chunk is 2^10 as in the forward kernel
int read_minors_opts(const perm_opts* o, int* prec, int* chunk, int* grid) {
  *prec = o ? o->prec : PERM_FP64;
  if (*prec != PERM_FP64 && *prec != PERM_FP64_DF && *prec != PERM_FP32X2) return PERM_EINVAL;
  if (o && o->block != 0 && o->block != MINORS_BLOCK) return PERM_EINVAL;
  *chunk = (o && o->chunk_log2) ? o->chunk_log2 : (*prec == PERM_FP32X2 ? 10 : 12);
  if (*chunk < 1 || *chunk > 30) return PERM_EINVAL;
  *grid = o ? o->grid : 0;
  if (*grid < 0) return PERM_EINVAL;
  return PERM_OK;
}

// Blocks per item: enough lanes for >= 64 Gray indices each, and no more than a
// resident wave shared by all items (opts->grid, when set, fixes it).
int plan_minors(int k, long long items, const perm_opts* o, MinorsPlan* p) {
  int prec, chunk, grid;
  int st = read_minors_opts(o, &prec, &chunk, &grid);
  if (st) return st;
  const uint64_t T = 1ull << (k - 1);
  long long bpi;
  if (grid > 0) {
    bpi = grid;
  } else {
    long long wave = 0;
    st = minors_wave(k, prec, &wave);
    if (st) return st;
    const long long by_work = (long long)((T + 64ull * MINORS_BLOCK - 1) / (64ull * MINORS_BLOCK));
    const long long by_wave = (wave + items - 1) / items;
    bpi = by_work < by_wave ? by_work : by_wave;
    if (bpi < 1) bpi = 1;
  }
  if (items * bpi > INT_MAX) return PERM_EINVAL;
  p->bpi = (int)bpi;
  p->chunk_log2 = chunk;
  p->prec = prec;
  const uint64_t lanes = (uint64_t)bpi * MINORS_BLOCK;
  p->per_q = T / lanes;
  p->per_r = T % lanes;
  return PERM_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct RowMinorsLayout {
  MinorsPlan plan;
  size_t scale_exp, partials, total;
};

int row_minors_layout(int k, int batch, const perm_opts* o, RowMinorsLayout* L) {
  int st = plan_minors(k, batch, o, &L->plan);
  if (st) return st;
  size_t off = 0;
  L->scale_exp = off;
  off = align256(off + sizeof(int) * (size_t)batch);
  L->partials = off;
  off = align256(off + (size_t)batch * L->plan.bpi * k * 4 * sizeof(double));
  L->total = off;
  return PERM_OK;
}

struct SampleLayout {
  size_t cmap, status, w, cum, partials, total;
};

int sample_layout(int m, int n, int nsamples, const perm_opts* o, SampleLayout* L) {
  size_t part = 0;
  for (int k = 2; k <= n; k++) {
    MinorsPlan p;
    int st = plan_minors(k, nsamples, o, &p);
    if (st) return st;
    const size_t b = (size_t)nsamples * p.bpi * k * 4 * sizeof(double);
    if (b > part) part = b;
  }
  size_t off = 0;
  L->cmap = off;
  off = align256(off + sizeof(int) * (size_t)nsamples * n);
  L->status = off;
  off = align256(off + sizeof(int) * (size_t)nsamples);
  L->w = off;
  off = align256(off + sizeof(double) * (size_t)nsamples * m);
  L->cum = off;
  off = align256(off + sizeof(double) * (size_t)nsamples * m);
  L->partials = off;
  off = align256(off + part);
  L->total = off;
  return PERM_OK;
}

}  // namespace

extern "C" {

size_t perm_row_minors_workspace_size(int k, int batch, const perm_opts* opts) {
  if (k < 1 || k > PERM_MINORS_MAX_K || batch < 0) return 0;
  if (k == 1 || batch == 0) return 256;
  RowMinorsLayout L;
  if (row_minors_layout(k, batch, opts, &L)) return 0;
  return L.total;
}

int perm_row_minors(const perm_c128* dM, int k, int ldm, int batch, int64_t strideM, perm_c128* dOut,
                    void* dWork, size_t workBytes, const perm_opts* opts, void* stream) {
  permk::NvtxRange nvtx_range("perm_row_minors");
  cudaStream_t s = (cudaStream_t)stream;
  if (k < 1 || k > PERM_MINORS_MAX_K) return PERM_ERANGE;
  if (batch < 0) return PERM_EINVAL;
  if (batch == 0) return PERM_OK;
  if (!dOut || ((uintptr_t)dOut & 15u)) return PERM_EINVAL;
  if (k == 1) {
    minors_one_kernel<<<(batch + 127) / 128, 128, 0, s>>>((double2*)dOut, batch);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PERM_OK : sfail((int)e);
  }
  if (!dM || ((uintptr_t)dM & 15u) || ldm < k) return PERM_EINVAL;
  if (batch > 1 && strideM < (int64_t)(k - 2) * ldm + k) return PERM_EINVAL;
  RowMinorsLayout L;
  int st = row_minors_layout(k, batch, opts, &L);
  if (st) return st;
  if (!dWork || ((uintptr_t)dWork & 255u)) return PERM_EINVAL;
  if (workBytes < L.total) return PERM_ENOMEM;
  char* w = (char*)dWork;
  MinorsArgs a;
  a.base = (const double2*)dM;
  a.rs = ldm;
  a.cs = 1;
  a.item_stride = batch > 1 ? strideM : 0;
  a.rows = nullptr;
  a.rows_stride = 0;
  a.cmap = nullptr;
  a.cmap_stride = 0;
  a.index_limit = INT_MAX;
  a.status = nullptr;
  a.bpi = L.plan.bpi;
  a.chunk_log2 = L.plan.chunk_log2;
  a.per_q = L.plan.per_q;
  a.per_r = L.plan.per_r;
  a.neg_zero = -0.0;
  a.partials = (double*)(w + L.partials);
  a.scale_exp = (int*)(w + L.scale_exp);
  int le = dispatch_minors(k, a, L.plan.prec, batch * L.plan.bpi, s);
  if (le) return sfail(le);
  MinorsReduceArgs r;
  r.partials = a.partials;
  r.bpi = L.plan.bpi;
  r.k = k;
  r.scale_exp = a.scale_exp;
  r.out = (double2*)dOut;
  minors_reduce_kernel<<<batch, 32, 0, s>>>(r);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PERM_OK : sfail((int)e);
}

size_t boson_sample_workspace_size(int m, int n, int nsamples, const perm_opts* opts) {
  if (n < 1 || n > BOSON_SAMPLE_MAX_N || m < n || nsamples < 0) return 0;
  if (nsamples == 0) return 256;
  SampleLayout L;
  if (sample_layout(m, n, nsamples, opts, &L)) return 0;
  return L.total;
}

int boson_sample(const perm_c128* dU, int m, int ldu, int n, const int32_t* hInputs, int nsamples,
                 const int32_t* dAlpha, const double* dUnif, int32_t* dR, void* dWork, size_t workBytes,
                 const perm_opts* opts, void* stream) {
  permk::NvtxRange nvtx_range("boson_sample");
  cudaStream_t s = (cudaStream_t)stream;
  if (n < 1 || n > BOSON_SAMPLE_MAX_N) return PERM_ERANGE;
  if (m < n || ldu < m || nsamples < 0 || !hInputs) return PERM_EINVAL;
  for (int j = 0; j < n; j++) {
    if (hInputs[j] < 0 || hInputs[j] >= m) return PERM_EINVAL;
    for (int i = 0; i < j; i++)
      if (hInputs[i] == hInputs[j]) return PERM_EINVAL;  // one photon per input mode
  }
  if (nsamples == 0) return PERM_OK;
  if (!dU || !dAlpha || !dUnif || !dR || ((uintptr_t)dU & 15u) || ((uintptr_t)dUnif & 7u) ||
      ((uintptr_t)dAlpha & 3u) || ((uintptr_t)dR & 3u))
    return PERM_EINVAL;
  SampleLayout L;
  int st = sample_layout(m, n, nsamples, opts, &L);
  if (st) return st;
  if (!dWork || ((uintptr_t)dWork & 255u)) return PERM_EINVAL;
  if (workBytes < L.total) return PERM_ENOMEM;
  char* w = (char*)dWork;
  int* cmap = (int*)(w + L.cmap);
  int* status = (int*)(w + L.status);

  SampleInitArgs ia;
  ia.n = n;
  ia.nsamples = nsamples;
  for (int j = 0; j < SAMPLE_MAX_N; j++) ia.inputs[j] = j < n ? hInputs[j] : 0;
  ia.alpha = dAlpha;
  ia.unif = dUnif;
  ia.cmap = cmap;
  ia.status = status;
  ia.R = dR;
  sample_init_kernel<<<(nsamples + 127) / 128, 128, 0, s>>>(ia);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return sfail((int)e);

  for (int k = 1; k <= n; k++) {
    MinorsPlan p{1, 12, 0, 0, 0};
    if (k >= 2) {
      st = plan_minors(k, nsamples, opts, &p);
      if (st) return st;
      MinorsArgs a;
      a.base = (const double2*)dU;
      a.rs = 1;       // M[i][j] = U[in(alpha_j)][r_i]: row index of M walks U's columns
      a.cs = ldu;
      a.item_stride = 0;
      a.rows = dR;
      a.rows_stride = n;
      a.cmap = cmap;
      a.cmap_stride = n;
      a.index_limit = m;
      a.status = status;
      a.bpi = p.bpi;
      a.chunk_log2 = p.chunk_log2;
      a.per_q = p.per_q;
      a.per_r = p.per_r;
      a.neg_zero = -0.0;
      a.partials = (double*)(w + L.partials);
      a.scale_exp = nullptr;
      int le = dispatch_minors(k, a, p.prec, nsamples * p.bpi, s);
      if (le) return sfail(le);
    }
    DrawArgs d;
    d.U = (const double2*)dU;
    d.ldu = ldu;
    d.m = m;
    d.n = n;
    d.k = k;
    d.cmap = cmap;
    d.unif = dUnif;
    d.R = dR;
    d.status = status;
    d.partials = (const double*)(w + L.partials);
    d.bpi = p.bpi;
    d.w = (double*)(w + L.w);
    d.cum = (double*)(w + L.cum);
    draw_kernel<<<nsamples, DRAW_BLOCK, 0, s>>>(d);
    e = cudaGetLastError();
    if (e != cudaSuccess) return sfail((int)e);
  }
  return PERM_OK;
}

}  // extern "C"
