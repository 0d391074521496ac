// Adjoint of the Glynn permanent in the same Gray-code pass (Supp. Eq. (S2)).
//
// dPer/da_ij = 2^-(n-1) sum_delta (prod delta) delta_j prod_{k != i} v_k(delta),
// v_i = sum_j delta_j a_ij.  With w_i = (prod delta) q_i, q_i = prod_{k != i} v_k,
// G_ij = sum over terms of w_i delta_j is accumulated at O(n) per term: S_i =
// running sum of w_i (shared memory) and H_ij = G_ij - delta_j S_i, which changes
// only when the Gray code flips column j (delta_j -> -delta_j): H_:j += 2
// delta_j^old S.  At the end G = H + delta S.
//
// Two adjacent lanes (a pair) share one Gray walk: the even lane owns rows
// 0..M-1, the odd lane rows M..n-1 (M = ceil(n/2); for odd n the odd lane's last
// row is a dummy with v = 1 that contributes nothing).  Each lane keeps its half
// of the row sums, of the suffix products, of S and of the prefetched H column,
// so the per-lane state is half that of one lane per walk and two warps fit on
// every SM sub-partition.  Per term a lane forms the suffix products of its rows
// down to its half's full product, swaps that product with its partner (one
// shuffle), and runs its prefix pass starting from (prod delta) x the partner's
// product: q_i = (prefix within the half) x (suffix within the half) x (the other
// half's product), no division (a row sum may be exactly zero).  Both lanes end
// with the whole term; both add it, and the forward sum is halved at the end.
// The per-pair H (n x n) lives in the caller's workspace, pair-interleaved so a
// warp's access is coalesced; a second kernel sums the pairs in a fixed order.
#pragma once
#include "fwd_kernel.cuh"

namespace permk {

constexpr int GRAD_MAX_N = 32;
constexpr int GRAD_BLOCK = 256;  // 128 lane pairs
// From this size on, the column of H that the next Gray step flips is prefetched
// into shared memory (cp.async) while the current term is computed, so its global
// latency (the per-pair state is far larger than L2) hides behind the term's FP64
// work.
constexpr int GRAD_PREFETCH_MIN_N = 16;

// rows per lane and the column stride of the staged matrix (room for the dummy row n)
template <int N>
struct GradShape {
  static constexpr int M = (N + 1) / 2;
  static constexpr int NP = (N + 1) | 1;
};

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

struct GradArgs {
  const double2* A;
  int lda;
  int chunk_log2;
  uint64_t per_q, per_r;  // floor/ceil split of the 2^(n-1) Gray indices over the lane pairs
  double neg_zero;
  double2* state;         // H: [i*N + j][P]
  long long P;            // lane pairs in the grid (= state stride)
  double* partials;       // forward Per (twice): 4 doubles per block
  int* scale_exp;         // [1 + N]: sum_i s_i, then s_i (written by block 0)
};

// Stores column 0 and the doubled columns 2 a_{:,b+1} (rows scaled by 2^{s_i})
// with column stride NP, plus a dummy row n (column 0 = 1, doubled columns 0) so
// that its row sum is exactly 1.  Returns sum_i s_i over the real rows.
template <int N>
__device__ int stage_matrix_doubled(const double2* __restrict__ A, int lda, double2* Col0, double2* Step,
                                    int* s_row) {
  constexpr int NP = GradShape<N>::NP;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    double nrm = 0.0;
    for (int j = 0; j < N; j++) {
      const double2 v = A[(size_t)i * lda + j];
      nrm = fma(v.x, v.x, nrm);
      nrm = fma(v.y, v.y, nrm);
    }
    const int e2 = (int)((__double2hiint(nrm) >> 20) & 0x7FF) - 1023;
    int s = (nrm == 0.0) ? 0 : -(e2 >> 1);
    s = s > 1000 ? 1000 : (s < -1000 ? -1000 : s);
    s_row[i] = s;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    const int i = idx / N, j = idx % N;
    const double f = pow2_double(s_row[i]);
    const double2 v = A[(size_t)i * lda + j];
    if (j == 0) Col0[i] = make_double2(v.x * f, v.y * f);
    else Step[(j - 1) * NP + i] = make_double2(2.0 * (v.x * f), 2.0 * (v.y * f));
  }
  if (threadIdx.x == 0) Col0[N] = make_double2(1.0, 0.0);
  for (int b = threadIdx.x; b < N - 1; b += blockDim.x) Step[b * NP + N] = make_double2(0.0, 0.0);
  int total = 0;
  for (int i = 0; i < N; i++) total += s_row[i];
  __syncthreads();
  return total;
}

template <int N>
__device__ __forceinline__ double2* hstate(const GradArgs& a, int i, int j, long long p) {
  return a.state + (long long)(i * N + j) * a.P + p;
}

// PREC 0: FP64 throughout; PREC 3 (R3): the prefix / suffix / q products in
// double-float on the FP32 pipe, row sums, S, H and the accumulation in FP64.
template <int N, int PREC>
__global__ void __launch_bounds__(GRAD_BLOCK, 1) grad_kernel(GradArgs a) {
  extern __shared__ double2 smem[];
  constexpr int M = GradShape<N>::M;
  constexpr int NP = GradShape<N>::NP;
  constexpr bool PF = (N >= GRAD_PREFETCH_MIN_N);
  // column 0 of A (plus the dummy row), then the doubled columns 2 a_{:,b+1}
  // (b = 0..N-2); the row sums at a chunk start are (2 a_{:,0} + sum_b +-2 a_{:,b+1})
  // / 2, exact.
  double2* Col0 = smem;
  double2* Step = smem + NP;
  const int B = blockDim.x;
  double2* suf = smem + N * NP + threadIdx.x;                // suf[r * B], r = 1..M-1
  double2* S = smem + N * NP + M * B + threadIdx.x;          // S[r * B]
  double2* Hbuf = smem + N * NP + 2 * M * B + threadIdx.x;   // Hbuf[r * B] (PF only)
  __shared__ int s_row[N];
  __shared__ dd wsum[2][GRAD_BLOCK / 32];

  const int scale_exp = stage_matrix_doubled<N>(a.A, a.lda, Col0, Step, s_row);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.scale_exp[0] = scale_exp;
    for (int i = 0; i < N; i++) a.scale_exp[1 + i] = s_row[i];
  }
  const double nz = a.neg_zero;
  const long long T = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long p = T >> 1;             // the pair
  const int half = (int)(T & 1);
  const int rb = half ? M : 0;            // global row of local row 0
  const int nvalid = half ? N - M : M;    // local rows that are real (the rest: the dummy row)
  const unsigned pair_mask = 3u << (threadIdx.x & 30);
  const uint64_t kb = a.per_q * (uint64_t)p + ((uint64_t)p < a.per_r ? (uint64_t)p : a.per_r);
  const uint64_t ke = kb + a.per_q + ((uint64_t)p < a.per_r ? 1 : 0);
  const uint64_t CH = 1ull << a.chunk_log2;

  // per-lane state starts at zero
  for (int r = 0; r < M; r++) {
    S[r * B] = make_double2(0.0, 0.0);
    if (r < nvalid)
      for (int j = 0; j < N; j++) *hstate<N>(a, rb + r, j, p) = make_double2(0.0, 0.0);
  }

  double ar = 0.0, ai = 0.0;
  uint64_t k = kb;
  uint64_t g = kb ^ (kb >> 1);
  while (k < ke) {
    const uint64_t c1 = (ke - k > CH) ? k + CH : ke;
    double vr[M], vi[M];
#pragma unroll
    for (int r = 0; r < M; r++) {
      const double2 x = Col0[rb + r];
      vr[r] = x.x + x.x;
      vi[r] = x.y + x.y;
    }
#pragma unroll 1
    for (int b = 0; b < N - 1; b++) {
      const double coef = ((g >> b) & 1ull) ? -1.0 : 1.0;
      const double2* col = Step + b * NP + rb;
#pragma unroll
      for (int r = 0; r < M; r++) {
        const double2 x = col[r];
        vr[r] = fma(coef, x.x, vr[r]);
        vi[r] = fma(coef, x.y, vi[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < M; r++) {
      vr[r] *= 0.5;
      vi[r] *= 0.5;
    }
#pragma unroll 1
    while (true) {
      if (PF && k + 1 < ke) {
        // the next step flips column ctz(k+1)+1: fetch this lane's rows of its H
        // while the term is computed
        const int bn = __ffsll((long long)(k + 1)) - 1;
        for (int r = 0; r < M; r++)
          if (r < nvalid) cp_async16(Hbuf + r * B, hstate<N>(a, rb + r, bn + 1, p));
        cp_async_commit();
      }
      const unsigned long long smask = (k & 1ull) << 63;  // (prod delta) = (-1)^(k & 1)
      if constexpr (PREC == 3) {
        // the products in double-float on the FP32 pipe (each FP64 row sum split
        // into two FP32 halves, ~48 bits); S, the flips and the row sums stay FP64
        df dr[M], di[M];
#pragma unroll
        for (int r = 0; r < M; r++) {
          dr[r] = f64_to_df(vr[r]);
          di[r] = f64_to_df(vi[r]);
        }
        float4* sufF = reinterpret_cast<float4*>(suf);
        df pr = dr[M - 1], pi = di[M - 1];
        if (M > 1) sufF[(M - 1) * B] = make_float4(pr.h, pr.l, pi.h, pi.l);
#pragma unroll
        for (int r = M - 2; r >= 1; r--) {
          dfc_mul(pr, pi, dr[r], di[r]);
          sufF[r * B] = make_float4(pr.h, pr.l, pi.h, pi.l);
        }
        if (M > 1) dfc_mul(pr, pi, dr[0], di[0]);
        const unsigned fs = (unsigned)(k & 1ull) << 31;  // the term's sign on FP32 bit patterns
        df er{__uint_as_float(__float_as_uint(__shfl_xor_sync(pair_mask, pr.h, 1)) ^ fs),
              __uint_as_float(__float_as_uint(__shfl_xor_sync(pair_mask, pr.l, 1)) ^ fs)};
        df ei{__uint_as_float(__float_as_uint(__shfl_xor_sync(pair_mask, pi.h, 1)) ^ fs),
              __uint_as_float(__float_as_uint(__shfl_xor_sync(pair_mask, pi.l, 1)) ^ fs)};
#pragma unroll
        for (int r = 0; r < M - 1; r++) {
          const float4 sf = sufF[(r + 1) * B];
          df tr = er, ti = ei;
          dfc_mul(tr, ti, df{sf.x, sf.y}, df{sf.z, sf.w});
          double2 si = S[r * B];
          si.x += f32_to_f64_int(tr.h) + f32_to_f64_int(tr.l);
          si.y += f32_to_f64_int(ti.h) + f32_to_f64_int(ti.l);
          S[r * B] = si;
          dfc_mul(er, ei, dr[r], di[r]);
        }
        double2 sl = S[(M - 1) * B];
        sl.x += f32_to_f64_int(er.h) + f32_to_f64_int(er.l);
        sl.y += f32_to_f64_int(ei.h) + f32_to_f64_int(ei.l);
        S[(M - 1) * B] = sl;
        dfc_mul(er, ei, dr[M - 1], di[M - 1]);
        ar += f32_to_f64_int(er.h) + f32_to_f64_int(er.l);
        ai += f32_to_f64_int(ei.h) + f32_to_f64_int(ei.l);
      } else {
        // suffix products of the half, suf_r = v_r ... v_{M-1}, down to the half's product
        double pr = vr[M - 1], pi = vi[M - 1];
        if (M > 1) suf[(M - 1) * B] = make_double2(pr, pi);
#pragma unroll
        for (int r = M - 2; r >= 1; r--) {
          cmul_inplace<3>(pr, pi, vr[r], vi[r], nz);
          suf[r * B] = make_double2(pr, pi);
        }
        if (M > 1) cmul_inplace<3>(pr, pi, vr[0], vi[0], nz);
        // the partner's half product; the prefix chain starts from (prod delta) x it,
        // so S_r += (prod delta) q_r = e suf_{r+1} is one complex multiply-add
        const double opr = __shfl_xor_sync(pair_mask, pr, 1);
        const double opi = __shfl_xor_sync(pair_mask, pi, 1);
        double er = xor_sign(opr, smask), ei = xor_sign(opi, smask);
#pragma unroll
        for (int r = 0; r < M - 1; r++) {
          const double2 sf = suf[(r + 1) * B];
          double2 si = S[r * B];
          si.x = fma(er, sf.x, si.x);
          si.x = fma(-ei, sf.y, si.x);
          si.y = fma(er, sf.y, si.y);
          si.y = fma(ei, sf.x, si.y);
          S[r * B] = si;
          cmul_inplace<3>(er, ei, vr[r], vi[r], nz);
        }
        // the half's last row: q = e
        double2 sl = S[(M - 1) * B];
        sl.x += er;
        sl.y += ei;
        S[(M - 1) * B] = sl;
        // the whole term (prod delta) prod_i v_i = e v_{M-1}, added by both lanes
        ar = fma(er, vr[M - 1], ar);
        ar = fma(-ei, vi[M - 1], ar);
        ai = fma(er, vi[M - 1], ai);
        ai = fma(ei, vr[M - 1], ai);
      }
      ++k;
      if (k >= ke) break;
      // column j = b+1 flips (delta_j -> -delta_j): H_:j += 2 delta_j^old S
      const int b = __ffsll((long long)k) - 1;
      const double f = xor_sign(2.0, ((g >> b) & 1ull) << 63);
      if (PF) cp_async_wait_all();
#pragma unroll
      for (int r = 0; r < M; r++) {
        if (r < nvalid) {
          const double2 sv = S[r * B];
          double2* hp = hstate<N>(a, rb + r, b + 1, p);
          double2 h = PF ? Hbuf[r * B] : *hp;
          h.x = fma(f, sv.x, h.x);
          h.y = fma(f, sv.y, h.y);
          *hp = h;
        }
      }
      g ^= 1ull << b;
      if (k >= c1) break;  // next chunk: recompute the row sums from g
      // bit now set: delta_{b+2} became -1, subtract 2a; bit now clear: add
      const double su = xor_sign(1.0, ((g >> b) & 1ull) << 63);
      const double2* col = Step + b * NP + rb;
#pragma unroll
      for (int r = 0; r < M; r++) {
        const double2 x = col[r];
        vr[r] = fma(su, x.x, vr[r]);
        vi[r] = fma(su, x.y, vi[r]);
      }
    }
  }
  // G = H + delta S with every column's current sign (column 0 is always +1)
  for (int j = 0; j < N; j++) {
    const double f = xor_sign(1.0, (j == 0) ? 0ull : (((g >> (j - 1)) & 1ull) << 63));
    for (int r = 0; r < nvalid; r++) {
      const double2 sv = S[r * B];
      double2* hp = hstate<N>(a, rb + r, j, p);
      double2 h = *hp;
      h.x = fma(f, sv.x, h.x);
      h.y = fma(f, sv.y, h.y);
      *hp = h;
    }
  }

  // forward permanent (every term added by both lanes of its pair): block partials
  dd sr{ar, 0.0}, si{ai, 0.0};
  warp_sum_dd(sr, si);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    wsum[0][warp] = sr;
    wsum[1][warp] = si;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    dd br = wsum[0][0], bi = wsum[1][0];
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
      br = dd_add(br, wsum[0][w]);
      bi = dd_add(bi, wsum[1][w]);
    }
    double* q = a.partials + 4 * (size_t)blockIdx.x;
    q[0] = br.hi;
    q[1] = br.lo;
    q[2] = bi.hi;
    q[3] = bi.lo;
  }
}

struct GradReduceArgs {
  const double2* state;
  long long P;
  int n;
  const double* partials;
  int nblocks;
  const int* scale_exp;  // [1 + n]
  double2* perm;         // nullable: Per
  double2* minor;        // nullable: dPer/da_ij, row-major n x n
  double2* grad_abs2;    // nullable: 2 Per conj(dPer/da_ij)
  double* abs2;          // nullable: |Per|^2
};

template <int N>
int launch_grad(const GradArgs& a, int prec, int grid, cudaStream_t s);
template <int N>
int grad_blocks_per_sm(int prec, int* out);

// dynamic shared memory: the staged matrix (n columns of stride NP), then per lane
// the half's suffix products, S and (n >= 16) the prefetched H column
inline size_t grad_smem_bytes(int N) {
  const int M = (N + 1) / 2, NP = (N + 1) | 1;
  const int bufs = N >= GRAD_PREFETCH_MIN_N ? 3 : 2;
  return (size_t)N * NP * sizeof(double2) + (size_t)bufs * M * GRAD_BLOCK * sizeof(double2);
}

}  // namespace permk
