// Gray-code Glynn / Ryser permanent kernels for sm_103a.
//
// One thread walks one contiguous piece of Gray indices (the per-process index
// range of Algorithms 1 and 2 of arXiv 1606.05836, here per thread).  Its n
// complex row sums live in registers; at every chunk start they are recomputed
// exactly from the matrix (Supp. Eq. (S1)/(S2) applied to that index), and in
// between each step adds or subtracts the one column whose bit the Gray code
// flips.  The n-way complex product and its signed accumulation follow, then a
// warp-shuffle / block / last-block grid reduction in double-double.
//
// The per-term work and the walk itself live in common.cuh (shared with the
// batched kernel).
#pragma once
#include "common.cuh"

namespace permk {

struct FwdArgs {
  const double2* A;  // row-major, a[i][j] = A[i*lda + j]
  int n;
  int lda;
  int kind;         // KIND_GLYNN / KIND_RYSER
  int chunk_log2;   // recompute the row sums every 2^chunk_log2 steps
  uint64_t k_begin; // Gray index range [k_begin, k_end)
  uint64_t k_end;
  uint64_t per_q;   // thread T walks [k_begin + T*per_q + min(T, per_r), ...): floor/ceil split
  uint64_t per_r;
  double neg_zero;  // -0.0, read at run time (keeps FMA-with-zero from folding)
  double* partials; // 4 doubles per block: re.hi, re.lo, im.hi, im.lo
  unsigned* ticket; // zero before launch; reset to zero by the last block
  double2* out;     // raw == 0: one value, the permanent; raw == 1: (hi, lo) partial sum
  int raw;
  // KIND_GLYNN_MULT only: A holds the g distinct columns (n x g, lda); the Gray
  // range runs over (class, free index) pairs, K = class * 2^nfree + free index.
  MultInfo mult;
};

// ---------------------------------------------------------------------------
// staging (step a1): matrix -> shared memory, column-major, rows scaled by 2^s_i
// ---------------------------------------------------------------------------

// Column stride in shared memory: odd, so lanes reading different columns at the
// same row hit different banks.
template <int N>
struct Stride {
  static constexpr int value = N | 1;
};

// Column-major layout: Acol[j*NP + i] = a_ij * 2^{s_i}; Step[b*NP + i] is the column
// that flips with Gray bit b (Glynn: 2 a_{i,b+1}; Ryser: a_{i,b}).  Rows are
// scaled by powers of two so that ||row_i||_2 lies in [1/2, 2): exact in FP64
// (no rounding), and it keeps FP32 products of the R2 rung inside FP32's
// exponent range.  Returns sum_i s_i (identical in every block).
template <int N>
__device__ int stage_matrix(const double2* __restrict__ A, int lda, int kind, double2* Acol, double2* Step,
                            int* s_row, double2* Xb = nullptr) {
  const int n = N;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double nrm = 0.0;
    for (int j = 0; j < n; j++) {
      const double2 v = A[(size_t)i * lda + j];
      nrm = fma(v.x, v.x, nrm);
      nrm = fma(v.y, v.y, nrm);
    }
    int e2 = (int)((__double2hiint(nrm) >> 20) & 0x7FF) - 1023;  // floor(log2 |row|^2) for normal values
    int s = (nrm == 0.0) ? 0 : -(e2 >> 1);
    s = s > 1000 ? 1000 : (s < -1000 ? -1000 : s);
    s_row[i] = s;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx % n;
    const double f = pow2_double(s_row[i]);
    const double2 v = A[(size_t)i * lda + j];
    Acol[j * Stride<N>::value + i] = make_double2(v.x * f, v.y * f);
  }
  __syncthreads();
  if (kind == KIND_GLYNN) {
    for (int idx = threadIdx.x; idx < (n - 1) * n; idx += blockDim.x) {
      const int b = idx / n, i = idx % n;
      const double2 v = Acol[(b + 1) * Stride<N>::value + i];
      Step[b * Stride<N>::value + i] = make_double2(v.x + v.x, v.y + v.y);
    }
  } else if (kind == KIND_RYSER_NW && Xb != nullptr) {
    // x_i = a_{i,n-1} - (1/2) sum_j a_ij, summed in column order
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double sr = 0.0, si = 0.0;
      for (int j = 0; j < n; j++) {
        const double2 v = Acol[j * Stride<N>::value + i];
        sr += v.x;
        si += v.y;
      }
      const double2 last = Acol[(n - 1) * Stride<N>::value + i];
      Xb[i] = make_double2(last.x - 0.5 * sr, last.y - 0.5 * si);
    }
  }
  int total = 0;
  for (int i = 0; i < n; i++) total += s_row[i];
  __syncthreads();
  return total;
}

// Staging for KIND_GLYNN_MULT: rows scaled by 2^{s_i} from the norms of the g
// distinct columns; all distinct columns to Acol, the free ones doubled to Step.
template <int N>
__device__ int stage_matrix_mult(const FwdArgs& a, double2* Acol, double2* Step, int* s_row) {
  constexpr int NP = Stride<N>::value;
  const int g = a.mult.g;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    double nrm = 0.0;
    for (int c = 0; c < g; c++) {
      const double2 v = a.A[(size_t)i * a.lda + c];
      nrm = fma(v.x, v.x, nrm);
      nrm = fma(v.y, v.y, nrm);
    }
    const int e2 = (int)((__double2hiint(nrm) >> 20) & 0x7FF) - 1023;
    int s = (nrm == 0.0) ? 0 : -(e2 >> 1);
    s = s > 1000 ? 1000 : (s < -1000 ? -1000 : s);
    s_row[i] = s;
    const double f = pow2_double(s);
    for (int c = 0; c < g; c++) {
      const double2 v = a.A[(size_t)i * a.lda + c];
      const double br = v.x * f, bi = v.y * f;
      Acol[c * NP + i] = make_double2(br, bi);
      const int role = a.mult.role[c];
      if (role >= 0) Step[role * NP + i] = make_double2(br + br, bi + bi);
    }
  }
  __syncthreads();
  int total = 0;
  for (int i = 0; i < N; i++) total += s_row[i];
  __syncthreads();
  return total;
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------

template <int N, int PREC, int TUNE>
__global__ void __launch_bounds__(256, 1) fwd_kernel(FwdArgs a) {
  extern __shared__ double2 smem[];
  double2* Acol = smem;
  constexpr int NP = Stride<N>::value;
  double2* Step = (a.kind == KIND_GLYNN || a.kind == KIND_GLYNN_MULT) ? smem + N * NP : smem;
  double2* Xb = smem + N * NP;  // Ryser-NW base vector (the otherwise unused second half)
  __shared__ int s_row[N];

  const int scale_exp = (a.kind == KIND_GLYNN_MULT) ? stage_matrix_mult<N>(a, Acol, Step, s_row)
                                                    : stage_matrix<N>(a.A, a.lda, a.kind, Acol, Step, s_row, Xb);
  const double nz = a.neg_zero;

  const uint64_t T = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t kb = a.k_begin + T * a.per_q + (T < a.per_r ? T : a.per_r);
  const uint64_t ke = kb + a.per_q + (T < a.per_r ? 1 : 0);
  const uint64_t CH = 1ull << a.chunk_log2;
  const bool glynn = (a.kind == KIND_GLYNN);

  double ar = 0.0, ai = 0.0, cr = 0.0, ci = 0.0;  // accumulator and (R1/R2) compensation

  dd sr, si;
  if constexpr (PREC == 4) {
    // R4 (Glynn only): the doubled columns to double-float, in place (16 bytes each)
    float4* StepF = reinterpret_cast<float4*>(Step);
    for (int idx = threadIdx.x; idx < (N - 1) * N; idx += blockDim.x) {
      const int b = idx / N, i = idx % N;
      const double2 v = Step[b * NP + i];
      const df re = f64_to_df(v.x), im = f64_to_df(v.y);
      StepF[b * NP + i] = make_float4(re.h, re.l, im.h, im.l);
    }
    __syncthreads();
    walk_range_df<N>(Acol, StepF, NP, kb, ke, CH, ar, ai);
    sr = dd{ar, 0.0};
    si = dd{ai, 0.0};
  } else if (a.kind == KIND_GLYNN_MULT && a.mult.nfree >= 5 && a.k_begin == 0) {
    // Warp-aligned split: each class's 2^nfree local indices are laid out
    // lane-major (lane l owns [l F, (l+1) F), F = 2^(nfree-5)), and warp w takes
    // a contiguous run of the class-by-class offsets o in [0, F).  All 32 lanes
    // of a warp then walk equal-length ranges of the same class and cross class
    // boundaries together (no lane restarts a chunk while the others wait), and
    // every lane's share differs by at most one term.
    sr = dd{0.0, 0.0};
    si = dd{0.0, 0.0};
    const int nfree = a.mult.nfree;
    const uint64_t F = 1ull << (nfree - 5);
    const uint64_t U = a.k_end >> 5;  // class-by-class offsets: classes x F
    const uint64_t W = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t w = T >> 5;
    const uint64_t lane = T & 31u;
    const uint64_t q = U / W, r = U % W;
    uint64_t u = w * q + (w < r ? w : r);
    const uint64_t u1 = u + q + (w < r ? 1 : 0);
    while (u < u1) {
      const uint64_t c = u >> (nfree - 5);
      const uint64_t ob = u - (c << (nfree - 5));
      const uint64_t oe = (u1 - (c << (nfree - 5)) < F) ? u1 - (c << (nfree - 5)) : F;
      const uint64_t base = (c << nfree) + lane * F;
      walk_range<N, PREC, TUNE, false>(Acol, Step, nullptr, &a.mult, &sr, &si, NP, a.kind, base + ob, base + oe, CH,
                                       nz, ar, ai, cr, ci);
      u = (c << (nfree - 5)) + oe;
    }
  } else if (a.kind == KIND_GLYNN_MULT) {
    sr = dd{0.0, 0.0};
    si = dd{0.0, 0.0};
    walk_range<N, PREC, TUNE, false>(Acol, Step, nullptr, &a.mult, &sr, &si, NP, a.kind, kb, ke, CH, nz, ar, ai, cr,
                                     ci);
  } else {
    walk_range<N, PREC, TUNE, false>(Acol, Step, Xb, nullptr, nullptr, nullptr, NP, a.kind, kb, ke, CH, nz, ar, ai,
                                     cr, ci);
    acc_to_dd<PREC>(ar, ai, cr, ci, sr, si);
  }

  // ---- reduction (step a6): warp butterfly, block, last-block grid sum ------
  warp_sum_dd(sr, si);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  __shared__ dd wsum[2][8];
  if (lane == 0) {
    wsum[0][warp] = sr;
    wsum[1][warp] = si;
  }
  __syncthreads();
  __shared__ bool am_last;
  if (threadIdx.x == 0) {
    dd br = wsum[0][0], bi = wsum[1][0];
    for (int w = 1; w < nwarps; w++) {
      br = dd_add(br, wsum[0][w]);
      bi = dd_add(bi, wsum[1][w]);
    }
    double* p = a.partials + 4 * (size_t)blockIdx.x;
    p[0] = br.hi;
    p[1] = br.lo;
    p[2] = bi.hi;
    p[3] = bi.lo;
    __threadfence();
    const unsigned t = atomicAdd(a.ticket, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  if (warp == 0) {
    dd tr{0.0, 0.0}, ti{0.0, 0.0};
    for (int blk = lane; blk < (int)gridDim.x; blk += 32) {
      const volatile double* p = a.partials + 4 * (size_t)blk;
      tr = dd_add(tr, dd{p[0], p[1]});
      ti = dd_add(ti, dd{p[2], p[3]});
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      dd orr{__shfl_xor_sync(0xffffffffu, tr.hi, off), __shfl_xor_sync(0xffffffffu, tr.lo, off)};
      dd oii{__shfl_xor_sync(0xffffffffu, ti.hi, off), __shfl_xor_sync(0xffffffffu, ti.lo, off)};
      tr = dd_add(tr, orr);
      ti = dd_add(ti, oii);
    }
    if (lane == 0) {
      // undo the row scaling; Glynn divides by 2^(n-1); Ryser multiplies by (-1)^n
      // Ryser-NW: x 2 (-1)^(n-1)
      int e = -scale_exp;
      if (!a.raw && (glynn || a.kind == KIND_GLYNN_MULT)) e -= (N - 1);
      if (!a.raw && a.kind == KIND_RYSER_NW) e += 1;
      double neg = 1.0;
      if (!a.raw && a.kind == KIND_RYSER && (N & 1)) neg = -1.0;
      if (!a.raw && a.kind == KIND_RYSER_NW && ((N - 1) & 1)) neg = -1.0;
      tr.hi = ldexp(tr.hi, e) * neg;
      tr.lo = ldexp(tr.lo, e) * neg;
      ti.hi = ldexp(ti.hi, e) * neg;
      ti.lo = ldexp(ti.lo, e) * neg;
      if (a.raw) {
        a.out[0] = make_double2(tr.hi, ti.hi);
        a.out[1] = make_double2(tr.lo, ti.lo);
      } else {
        a.out[0] = make_double2(tr.hi + tr.lo, ti.hi + ti.lo);
      }
      *a.ticket = 0u;
    }
  }
}

// host-side launch helpers, explicitly instantiated per N in fwd_inst_*.cu
template <int N>
int launch_fwd(const FwdArgs& a, int prec, int tune, int grid, int block, cudaStream_t s);
template <int N>
int fwd_blocks_per_sm(int prec, int tune, int block, int kind, int* out);

inline size_t fwd_smem_bytes(int N, int kind) {
  const size_t cols = (kind == KIND_RYSER) ? (size_t)N : 2 * (size_t)N;
  return cols * (N | 1) * sizeof(double2);
}

}  // namespace permk
