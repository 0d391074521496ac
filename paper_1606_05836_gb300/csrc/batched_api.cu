// Batched permanents: the planner, prep and reduce kernels and the C ABI entry
// points perm_batched_workspace_size / perm_batched (declared in perm.h).
// The persistent walk kernel is in batched_kernel.cuh / batched_inst.cu.
#include <cuda_runtime.h>
#include <stdint.h>

#include "batched_kernel.cuh"
#include "host_util.h"
#include "perm.h"

namespace permk {

// Inclusive block scan (Hillis-Steele) of one int64 per thread.
__device__ inline long long block_scan_incl(long long v, long long* sh) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {
    long long add = (t >= off) ? sh[t - off] : 0;
    __syncthreads();
    sh[t] += add;
    __syncthreads();
  }
  long long r = sh[t];
  __syncthreads();
  return r;
}

// Per item (one warp each): bitwise-identical columns are one group; with any
// group of two or more copies (and use_mult) the item gets the column structure
// of the multiplicity expansion of Eq. (S2) — the delta = +1 copy from the first
// singleton group, else from the first smallest group; singletons are free
// columns, a group of m copies enters through its number k of -1 signs (radix
// m + 1, or m for the group holding the fixed copy) — and its index space is
// classes x 2^free.  Otherwise g = 0 and the index space is 2^M.
__global__ void __launch_bounds__(32) batch_mult_kernel(BatchArgs a) {
  const int lane = threadIdx.x;
  for (int item = blockIdx.x; item < a.count; item += gridDim.x) {
    const int n = a.ns[item];
    MultInfo* mi = a.mult + item;
    if (n < 1 || n > BATCH_MAX_N) {  // the planner reports it; keep the workspace sane
      if (lane == 0) {
        mi->g = 0;
        a.terms[item] = 1;
      }
      continue;
    }
    const double2* A = a.packed + a.offsets[item];
    int rep = lane;  // smallest column index with the same entries
    if (a.use_mult && lane < n) {
      for (int c = 0; c < lane; c++) {
        bool same = true;
        for (int i = 0; i < n && same; i++) {
          const double2 x = A[i * n + lane], y = A[i * n + c];
          same = (__double_as_longlong(x.x) == __double_as_longlong(y.x)) &&
                 (__double_as_longlong(x.y) == __double_as_longlong(y.y));
        }
        if (same) {
          rep = c;
          break;
        }
      }
    }
    __shared__ int reps[BATCH_MAX_N];
    reps[lane] = rep;
    __syncwarp();
    if (lane == 0) {
      int mult[BATCH_MAX_N], col[BATCH_MAX_N], g = 0;
      bool repeated = false;
      for (int j = 0; j < n; j++) {
        if (reps[j] == j) {
          col[g] = j;
          mult[g++] = 1;
        } else {
          for (int c = 0; c < g; c++)
            if (col[c] == reps[j]) {
              mult[c]++;
              repeated = true;
            }
        }
      }
      const int M = batch_M(n, a.kind);
      if (!a.use_mult || !repeated) {
        mi->g = 0;
        a.terms[item] = 1ll << M;
      } else {
        int fixed = -1;
        for (int c = 0; c < g && fixed < 0; c++)
          if (mult[c] == 1) fixed = c;
        if (fixed < 0) {
          fixed = 0;
          for (int c = 1; c < g; c++)
            if (mult[c] < mult[fixed]) fixed = c;
        }
        int nfree = 0;
        long long classes = 1;
        for (int c = 0; c < g; c++) {
          mi->mult[c] = (unsigned char)mult[c];
          mi->radix[c] = 0;
          mi->radix_base[c] = 1;
          if (mult[c] == 1) {
            mi->role[c] = (signed char)((c == fixed) ? -1 : nfree++);
          } else {
            mi->role[c] = -2;
            mi->radix[c] = (unsigned char)((c == fixed) ? mult[c] : mult[c] + 1);
            mi->radix_base[c] = classes;
            classes *= mi->radix[c];
          }
          a.mcol[item * BATCH_MAX_N + c] = (signed char)col[c];
        }
        mi->nfree = nfree;
        mi->g = g;
        a.terms[item] = classes << nfree;
      }
    }
    __syncwarp();
  }
}

__global__ void __launch_bounds__(BATCH_PLAN_THREADS) batch_plan_kernel(BatchArgs a) {
  __shared__ int hist[BATCH_MAX_N + 1];
  __shared__ int base[BATCH_MAX_N + 1];
  __shared__ long long sh[BATCH_PLAN_THREADS];
  __shared__ int bad;
  const int t = threadIdx.x, P = blockDim.x;
  if (t <= BATCH_MAX_N) hist[t] = 0;
  if (t == 0) bad = 0;
  __syncthreads();
  for (int i = t; i < a.count; i += P) {
    const int n = a.ns[i];
    if (n < 1 || n > BATCH_MAX_N) atomicOr(&bad, BATCH_BAD_N);
    else atomicAdd(&hist[n], 1);
  }
  __syncthreads();
  if (t == 0) {
    int run = 0;
    for (int n = BATCH_MAX_N; n >= 1; n--) {
      base[n] = run;
      run += hist[n];
    }
  }
  __syncthreads();
  if (bad) {
    if (t == 0) {
      *a.status = bad;
      *a.total_units = 0;
      *a.cursor = 0ull;
    }
    return;
  }
  for (int i = t; i < a.count; i += P) {
    const int p = atomicAdd(&base[a.ns[i]], 1);
    a.order[p] = i;
    a.pos[i] = p;
  }
  __syncthreads();
  // unit_start over sorted positions: each thread owns a contiguous segment
  const int seg = (a.count + P - 1) / P;
  const int lo = t * seg, hi = min(a.count, lo + seg);
  long long mine = 0;
  for (int p = lo; p < hi; p++) mine += batch_units(a.terms[a.order[p]], a.unit_log2);
  long long incl = block_scan_incl(mine, sh);
  long long run = incl - mine;
  for (int p = lo; p < hi; p++) {
    a.unit_start[p] = run;
    run += batch_units(a.terms[a.order[p]], a.unit_log2);
  }
  const long long total_units = sh[P - 1 < 0 ? 0 : P - 1];
  __syncthreads();
  // prep offsets by item index
  mine = 0;
  for (int i = lo; i < hi; i++) mine += batch_prep_elems(a.ns[i], a.kind);
  incl = block_scan_incl(mine, sh);
  run = incl - mine;
  for (int i = lo; i < hi; i++) {
    a.prep_off[i] = run;
    run += batch_prep_elems(a.ns[i], a.kind);
  }
  const long long total_prep = sh[P - 1];
  if (t == 0) {
    // block_scan_incl leaves the totals in sh[P-1] of each scan
    a.unit_start[a.count] = total_units;
    int st = BATCH_OK;
    if (total_units > a.units_cap || total_prep > a.prep_cap) st = BATCH_NO_ROOM;
    *a.status = st;
    *a.total_units = (st == BATCH_OK) ? total_units : 0;
    *a.cursor = 0ull;
  }
}

__global__ void __launch_bounds__(128) batch_prep_kernel(BatchArgs a) {
  __shared__ int s_row[BATCH_MAX_N];
  __shared__ int total;
  if (*a.status != BATCH_OK) return;
  for (int item = blockIdx.x; item < a.count; item += gridDim.x) {
    const int n = a.ns[item];
    const double2* A = a.packed + a.offsets[item];
    double2* C = a.prep + a.prep_off[item];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double nrm = 0.0;
      for (int j = 0; j < n; j++) {
        const double2 v = A[i * n + j];
        nrm = fma(v.x, v.x, nrm);
        nrm = fma(v.y, v.y, nrm);
      }
      const int e2 = (int)((__double2hiint(nrm) >> 20) & 0x7FF) - 1023;
      int s = (nrm == 0.0) ? 0 : -(e2 >> 1);
      s = s > 1000 ? 1000 : (s < -1000 ? -1000 : s);
      s_row[i] = s;
    }
    __syncthreads();
    const MultInfo* mi = a.mult + item;
    if (a.use_mult && mi->g > 0) {
      // repeated columns: the g distinct columns, then the doubled free ones by free index
      const int g = mi->g;
      for (int idx = threadIdx.x; idx < n * g; idx += blockDim.x) {
        const int i = idx % n, c = idx / n;
        const double f = pow2_double(s_row[i]);
        const double2 v = A[i * n + a.mcol[item * BATCH_MAX_N + c]];
        C[c * n + i] = make_double2(v.x * f, v.y * f);
        const int role = mi->role[c];
        if (role >= 0) C[n * n + role * n + i] = make_double2(2.0 * v.x * f, 2.0 * v.y * f);
      }
    } else {
      for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx % n, j = idx / n;
        const double f = pow2_double(s_row[i]);
        const double2 v = A[i * n + j];
        C[j * n + i] = make_double2(v.x * f, v.y * f);
        if (a.kind == KIND_GLYNN && j >= 1) {
          const double sr = 2.0 * v.x * f, si = 2.0 * v.y * f;
          if (a.prec == PERM_FP32X2) {
            // R4 walks add the step columns in double-float (16 bytes, same slot)
            const df re = f64_to_df(sr), im = f64_to_df(si);
            reinterpret_cast<float4*>(C)[n * n + (j - 1) * n + i] = make_float4(re.h, re.l, im.h, im.l);
          } else {
            C[n * n + (j - 1) * n + i] = make_double2(sr, si);
          }
        }
      }
    }
    if (threadIdx.x == 0) {
      int sum = 0;
      for (int i = 0; i < n; i++) sum += s_row[i];
      total = sum;
    }
    __syncthreads();
    if (threadIdx.x == 0) a.scale_exp[item] = total;
    __syncthreads();
  }
}

__global__ void batch_reduce_kernel(BatchArgs a) {
  const int item = blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= a.count) return;
  const int st = *a.status;
  if (st != BATCH_OK) {
    const double nan = __longlong_as_double(0x7FF8000000000000ll);
    a.out[item] = make_double2(nan, nan);
    if (a.prob) a.prob[item] = nan;
    return;
  }
  const int p = a.pos[item];
  const long long u0 = a.unit_start[p], u1 = a.unit_start[p + 1];
  dd tr{0.0, 0.0}, ti{0.0, 0.0};
  for (long long u = u0; u < u1; u++) {
    const double* q = a.partials + 4 * (size_t)u;
    tr = dd_add(tr, dd{q[0], q[1]});
    ti = dd_add(ti, dd{q[2], q[3]});
  }
  const int n = a.ns[item];
  const bool glynn = (a.kind == KIND_GLYNN);
  int e = -a.scale_exp[item];
  if (glynn) e -= (n - 1);
  const double neg = (!glynn && (n & 1)) ? -1.0 : 1.0;
  const double re = ldexp(tr.hi + tr.lo, e) * neg;
  const double im = ldexp(ti.hi + ti.lo, e) * neg;
  a.out[item] = make_double2(re, im);
  if (a.prob) {
    const double s = a.scale ? a.scale[item] : 1.0;
    a.prob[item] = fma(re, re, im * im) * s;
  }
}


}  // namespace permk

namespace {

using namespace permk;

int bfail(cudaError_t e) {
  record_cuda_error((int)e);
  return PERM_ECUDA;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  size_t cursor, status, total_units, order, pos, unit_start, prep_off, scale_exp, terms, mult, mcol, partials, prep,
      total;
  long long units_cap, prep_cap;
};

int batch_opts(const perm_opts* o, int* prec, int* chunk, int* unit, int* block, int* grid) {
  *prec = o ? o->prec : PERM_FP64;
  *chunk = (o && o->chunk_log2) ? o->chunk_log2 : ((o && o->prec == PERM_FP32X2) ? 10 : 12);
  *unit = (o && o->unit_log2) ? o->unit_log2 : 11;
  *block = (o && o->block) ? o->block : 128;
  *grid = o ? o->grid : 0;
  if (*prec < PERM_FP64 || *prec > PERM_FP32X2) return PERM_EINVAL;
  if (*chunk < 1 || *chunk > 30 || *unit < 0 || *unit > 30) return PERM_EINVAL;
  if (*block < 32 || *block > 256 || (*block & 31) || *grid < 0) return PERM_EINVAL;
  return PERM_OK;
}

int make_layout(int count, const int32_t* hN, int kind, int unit_log2, Layout* L) {
  long long units = 0, prep = 0;
  for (int i = 0; i < count; i++) {
    const int n = hN[i];
    if (n < 1 || n > BATCH_MAX_N) return PERM_ERANGE;
    units += batch_units(1ll << batch_M(n, kind), unit_log2);
    prep += batch_prep_elems(n, kind);
  }
  size_t off = 0;
  L->cursor = off; off += 8;
  L->status = off; off += 8;
  L->total_units = off; off += 8;
  off = align256(off);
  L->order = off; off = align256(off + 4 * (size_t)count);
  L->pos = off; off = align256(off + 4 * (size_t)count);
  L->unit_start = off; off = align256(off + 8 * ((size_t)count + 1));
  L->prep_off = off; off = align256(off + 8 * (size_t)count);
  L->scale_exp = off; off = align256(off + 4 * (size_t)count);
  L->terms = off; off = align256(off + 8 * (size_t)count);
  L->mult = off; off = align256(off + sizeof(MultInfo) * (size_t)count);
  L->mcol = off; off = align256(off + BATCH_MAX_N * (size_t)count);
  L->partials = off; off = align256(off + 32 * (size_t)units);
  L->prep = off; off = align256(off + 16 * (size_t)prep);
  L->total = off;
  L->units_cap = units;
  L->prep_cap = prep;
  return PERM_OK;
}

int walk_launch(int prec, const BatchArgs& a, int grid, int block, cudaStream_t s) {
  if (prec == 1) return launch_batch_walk<1>(a, grid, block, s);
  if (prec == 2) return launch_batch_walk<2>(a, grid, block, s);
  if (prec == 3) return launch_batch_walk<3>(a, grid, block, s);
  if (prec == 4) return launch_batch_walk<4>(a, grid, block, s);
  return launch_batch_walk<0>(a, grid, block, s);
}

int walk_occupancy(int prec, int block, int* out) {
  if (prec == 1) return batch_walk_blocks_per_sm<1>(block, out);
  if (prec == 2) return batch_walk_blocks_per_sm<2>(block, out);
  if (prec == 3) return batch_walk_blocks_per_sm<3>(block, out);
  if (prec == 4) return batch_walk_blocks_per_sm<4>(block, out);
  return batch_walk_blocks_per_sm<0>(block, out);
}

}  // namespace

extern "C" {

size_t perm_batched_workspace_size(int count, const int32_t* hN, int method, const perm_opts* opts) {
  int prec, chunk, unit, block, grid;
  if (count < 0 || (count > 0 && !hN) || (method != 0 && method != 1)) return 0;
  if (batch_opts(opts, &prec, &chunk, &unit, &block, &grid)) return 0;
  if (prec == PERM_FP32X2 && method != 0) return 0;  // R4 is a Glynn walk
  Layout L;
  if (make_layout(count, hN, method == 0 ? KIND_GLYNN : KIND_RYSER, unit, &L)) return 0;
  return L.total;
}

int perm_batched(const perm_c128* dPacked, const int64_t* dOffsets, const int32_t* dN, const int32_t* hN, int count,
                 int method, const double* dScale, perm_c128* dOut, double* dProb, void* dWork, size_t workBytes,
                 const perm_opts* opts, void* stream) {
  permk::NvtxRange nvtx_range("perm_batched");
  cudaStream_t s = (cudaStream_t)stream;
  if (count < 0 || (method != 0 && method != 1)) return PERM_EINVAL;
  if (count == 0) return PERM_OK;
  if (!dPacked || !dOffsets || !dN || !hN || !dOut || !dWork) return PERM_EINVAL;
  if (((uintptr_t)dPacked & 15u) || ((uintptr_t)dOut & 15u) || ((uintptr_t)dWork & 255u)) return PERM_EINVAL;
  int prec, chunk, unit, block, grid;
  int st = batch_opts(opts, &prec, &chunk, &unit, &block, &grid);
  if (st) return st;
  if (prec == PERM_FP32X2 && method != 0) return PERM_EINVAL;  // R4 is a Glynn walk
  const int kind = method == 0 ? KIND_GLYNN : KIND_RYSER;
  Layout L;
  st = make_layout(count, hN, kind, unit, &L);
  if (st) return st;
  if (workBytes < L.total) return PERM_ENOMEM;
  char* w = (char*)dWork;
  BatchArgs a;
  a.packed = (const double2*)dPacked;
  a.offsets = (const long long*)dOffsets;
  a.ns = (const int*)dN;
  a.count = count;
  a.kind = kind;
  a.prec = prec;
  a.unit_log2 = unit;
  a.chunk_log2 = chunk;
  a.neg_zero = -0.0;
  a.cursor = (unsigned long long*)(w + L.cursor);
  a.status = (int*)(w + L.status);
  a.total_units = (long long*)(w + L.total_units);
  a.order = (int*)(w + L.order);
  a.pos = (int*)(w + L.pos);
  a.unit_start = (long long*)(w + L.unit_start);
  a.prep_off = (long long*)(w + L.prep_off);
  a.scale_exp = (int*)(w + L.scale_exp);
  a.partials = (double*)(w + L.partials);
  a.terms = (long long*)(w + L.terms);
  a.mult = (MultInfo*)(w + L.mult);
  a.mcol = (signed char*)(w + L.mcol);
  // the expansion for R0-R2; the double-float rungs walk the expanded matrix
  // (their walk kernels carry no expansion branch: the R3 batch measured 0.396 s
  // with it against 0.370 s without)
  a.use_mult = (kind == KIND_GLYNN && prec != PERM_FP32X2 && prec != PERM_FP64_DF) ? 1 : 0;
  a.prep = (double2*)(w + L.prep);
  a.units_cap = L.units_cap;
  a.prep_cap = L.prep_cap;
  a.scale = dScale;
  a.out = (double2*)dOut;
  a.prob = dProb;
  if (grid <= 0) {
    int dev = 0, sms = 0, bps = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return bfail(e);
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return bfail(e);
    int oe = walk_occupancy(prec, block, &bps);
    if (oe) return bfail((cudaError_t)oe);
    if (bps < 1) return bfail(cudaErrorInvalidConfiguration);
    grid = sms * bps;
  }
  batch_mult_kernel<<<count < 4096 ? count : 4096, 32, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return bfail(e);
  batch_plan_kernel<<<1, BATCH_PLAN_THREADS, 0, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return bfail(e);
  const int prep_grid = count < 4096 ? count : 4096;
  batch_prep_kernel<<<prep_grid, 128, 0, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return bfail(e);
  int le = walk_launch(prec, a, grid, block, s);
  if (le) return bfail((cudaError_t)le);
  batch_reduce_kernel<<<(count + 127) / 128, 128, 0, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return bfail(e);
  return PERM_OK;
}

}  // extern "C"
