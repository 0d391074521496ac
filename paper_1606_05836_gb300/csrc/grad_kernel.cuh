// Adjoint of the Glynn permanent in the same Gray-code pass (Supp. Eq. (S2)).
//
// dPer/da_ij = 2^-(n-1) sum_delta (prod delta) delta_j prod_{k != i} v_k(delta),
// v_i = sum_j delta_j a_ij.  Per term, q_i = prod_{k != i} v_k comes from one
// suffix pass (stored per lane in shared memory) and one prefix pass — 2(n-2)
// complex multiplies plus one complex multiply-add per row that forms q_i and
// adds it to S_i at once, no division (a row sum may be exactly zero).  With
// w_i = (prod delta) q_i, G_ij = sum over terms of w_i delta_j is accumulated at
// O(n) per term: S_i = running sum of w_i (shared memory) and H_ij = G_ij -
// delta_j S_i, which changes only when the Gray code flips column j
// (delta_j -> -delta_j): H_:j += 2 delta_j^old S.  At the end G = H + delta S.
// The per-lane H (n x n) lives in the caller's workspace, lane-interleaved so
// every warp access is coalesced; a second kernel sums the lanes in a fixed order.
#pragma once
#include "fwd_kernel.cuh"

namespace permk {

constexpr int GRAD_MAX_N = 32;
constexpr int GRAD_BLOCK = 128;
// From this size on, the column of H that the next Gray step flips is prefetched
// into shared memory (cp.async) while the current term is computed, so its global
// latency (the per-lane state is far larger than L2) hides behind the term's FP64
// work.  The buffer costs occupancy (one block per SM from n = 20 on) and still
// wins: measured 1.54x at n = 20, 1.07x at n = 24, 1.53x at n = 32.
constexpr int GRAD_PREFETCH_MIN_N = 16;

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
  uint64_t per_q, per_r;  // floor/ceil split of the 2^(n-1) Gray indices over the lanes
  double neg_zero;
  double2* state;         // H: [i*N + j][P]
  long long P;            // lanes in the grid (= state stride)
  double* partials;       // forward Per: 4 doubles per block
  int* scale_exp;         // [1 + N]: sum_i s_i, then s_i (written by block 0)
};

// Like stage_matrix, but stores column 0 and the doubled columns 2 a_{:,b+1}
// only (rows scaled by 2^{s_i}).  Returns sum_i s_i.
template <int N>
__device__ int stage_matrix_doubled(const double2* __restrict__ A, int lda, double2* Col0, double2* Step,
                                    int* s_row) {
  constexpr int NP = Stride<N>::value;
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
  int total = 0;
  for (int i = 0; i < N; i++) total += s_row[i];
  __syncthreads();
  return total;
}

template <int N>
__device__ __forceinline__ double2* hstate(const GradArgs& a, int i, int j, long long T) {
  return a.state + (long long)(i * N + j) * a.P + T;
}

// H_:j += f S   (f = +-2 as a double: 2 delta_j^old at a flip, delta_j at the end)
template <int N>
__device__ __forceinline__ void flush_column(const GradArgs& a, int j, double f, const double2* S, int B,
                                             long long T) {
#pragma unroll 8
  for (int i = 0; i < N; i++) {
    const double2 s = S[i * B];
    double2* hp = hstate<N>(a, i, j, T);
    double2 h = *hp;
    h.x = fma(f, s.x, h.x);
    h.y = fma(f, s.y, h.y);
    *hp = h;
  }
}

template <int N>
__global__ void __launch_bounds__(GRAD_BLOCK, 1) grad_kernel(GradArgs a) {
  extern __shared__ double2 smem[];
  constexpr int NP = Stride<N>::value;
  // column 0 of A, then the doubled columns 2 a_{:,b+1} (b = 0..N-2); the row
  // sums at a chunk start are (2 a_{:,0} + sum_b +-2 a_{:,b+1}) / 2, exact.
  double2* Col0 = smem;
  double2* Step = smem + NP;
  const int B = blockDim.x;
  double2* suf = smem + N * NP + threadIdx.x;            // suf[i * B]
  double2* S = smem + N * NP + N * B + threadIdx.x;      // S[i * B]
  constexpr bool PF = (N >= GRAD_PREFETCH_MIN_N);
  double2* Hbuf = smem + N * NP + 2 * N * B + threadIdx.x;  // Hbuf[i * B] (PF only)
  __shared__ int s_row[N];
  __shared__ dd wsum[2][GRAD_BLOCK / 32];

  const int scale_exp = stage_matrix_doubled<N>(a.A, a.lda, Col0, Step, s_row);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.scale_exp[0] = scale_exp;
    for (int i = 0; i < N; i++) a.scale_exp[1 + i] = s_row[i];
  }
  const double nz = a.neg_zero;
  const long long T = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t kb = a.per_q * (uint64_t)T + ((uint64_t)T < a.per_r ? (uint64_t)T : a.per_r);
  const uint64_t ke = kb + a.per_q + ((uint64_t)T < a.per_r ? 1 : 0);
  const uint64_t CH = 1ull << a.chunk_log2;

  // per-lane state starts at zero
  for (int i = 0; i < N; i++) {
    S[i * B] = make_double2(0.0, 0.0);
    for (int j = 0; j < N; j++) *hstate<N>(a, i, j, T) = make_double2(0.0, 0.0);
  }

  double ar = 0.0, ai = 0.0;
  uint64_t k = kb;
  uint64_t g = kb ^ (kb >> 1);
  while (k < ke) {
    const uint64_t c1 = (ke - k > CH) ? k + CH : ke;
    double vr[N], vi[N];
#pragma unroll
    for (int i = 0; i < N; i++) {
      vr[i] = 0.0;
      vi[i] = 0.0;
    }
#pragma unroll
    for (int i = 0; i < N; i++) {
      const double2 x = Col0[i];
      vr[i] = x.x + x.x;
      vi[i] = x.y + x.y;
    }
#pragma unroll 1
    for (int b = 0; b < N - 1; b++) {
      const double coef = ((g >> b) & 1ull) ? -1.0 : 1.0;
      const double2* col = Step + b * NP;
#pragma unroll
      for (int i = 0; i < N; i++) {
        const double2 x = col[i];
        vr[i] = fma(coef, x.x, vr[i]);
        vi[i] = fma(coef, x.y, vi[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < N; i++) {
      vr[i] *= 0.5;
      vi[i] *= 0.5;
    }
#pragma unroll 1
    while (true) {
      if (PF && k + 1 < ke) {
        // the next step flips column ctz(k+1)+1: fetch its H while this term is computed
        const int bn = __ffsll((long long)(k + 1)) - 1;
        for (int i = 0; i < N; i++) cp_async16(Hbuf + i * B, hstate<N>(a, i, bn + 1, T));
        cp_async_commit();
      }
      const unsigned long long smask = (k & 1ull) << 63;  // (prod delta) = (-1)^(k & 1)
      const double sgn = xor_sign(1.0, smask);
      if (N == 1) {
        // q_0 = 1 (empty product); Per term = v_0
        double2 s0 = S[0];
        s0.x += sgn;
        S[0] = s0;
        ar = fma(sgn, vr[0], ar);
        ai = fma(sgn, vi[0], ai);
      } else {
        // suffix products suf_i = v_i ... v_{N-1}, i >= 1
        double pr = vr[N - 1], pi = vi[N - 1];
        suf[(N - 1) * B] = make_double2(pr, pi);
#pragma unroll
        for (int i = N - 2; i >= 1; i--) {
          cmul_inplace<3>(pr, pi, vr[i], vi[i], nz);
          suf[i * B] = make_double2(pr, pi);
        }
        // prefix pass, carrying the term's sign: e = (prod delta) v_0 ... v_{i-1}, so
        // S_i += (prod delta) q_i = e suf_{i+1} is one complex multiply-add (4 FMAs)
        double2 s0 = S[0];  // q_0 = suf_1
        s0.x = fma(sgn, pr, s0.x);
        s0.y = fma(sgn, pi, s0.y);
        S[0] = s0;
        double er = xor_sign(vr[0], smask), ei = xor_sign(vi[0], smask);
#pragma unroll
        for (int i = 1; i < N - 1; i++) {
          const double2 sf = suf[(i + 1) * B];
          double2 si = S[i * B];
          si.x = fma(er, sf.x, si.x);
          si.x = fma(-ei, sf.y, si.x);
          si.y = fma(er, sf.y, si.y);
          si.y = fma(ei, sf.x, si.y);
          S[i * B] = si;
          cmul_inplace<3>(er, ei, vr[i], vi[i], nz);
        }
        // q_{N-1} = prefix of all but the last row (e already carries the sign)
        double2 sl = S[(N - 1) * B];
        sl.x += er;
        sl.y += ei;
        S[(N - 1) * B] = sl;
        // forward term: (prod delta) * prefix * v_{N-1}
        ar = fma(er, vr[N - 1], ar);
        ar = fma(-ei, vi[N - 1], ar);
        ai = fma(er, vi[N - 1], ai);
        ai = fma(ei, vr[N - 1], ai);
      }
      ++k;
      if (k >= ke) break;
      // column j = b+1 flips (delta_j -> -delta_j): H_:j += 2 delta_j^old S
      const int b = __ffsll((long long)k) - 1;
      if (PF) {
        const double f = xor_sign(2.0, ((g >> b) & 1ull) << 63);
        cp_async_wait_all();
#pragma unroll 8
        for (int i = 0; i < N; i++) {
          const double2 sv = S[i * B];
          double2 h = Hbuf[i * B];
          h.x = fma(f, sv.x, h.x);
          h.y = fma(f, sv.y, h.y);
          *hstate<N>(a, i, b + 1, T) = h;
        }
      } else {
        flush_column<N>(a, b + 1, xor_sign(2.0, ((g >> b) & 1ull) << 63), S, B, T);
      }
      g ^= 1ull << b;
      if (k >= c1) break;  // next chunk: recompute the row sums from g
      // bit now set: delta_{b+2} became -1, subtract 2a; bit now clear: add
      const double su = xor_sign(1.0, ((g >> b) & 1ull) << 63);
      const double2* col = Step + b * NP;
#pragma unroll
      for (int i = 0; i < N; i++) {
        const double2 x = col[i];
        vr[i] = fma(su, x.x, vr[i]);
        vi[i] = fma(su, x.y, vi[i]);
      }
    }
  }
  // G = H + delta S with every column's current sign (column 0 is always +1)
  for (int j = 0; j < N; j++) {
    const unsigned long long neg = (j == 0) ? 0ull : (((g >> (j - 1)) & 1ull) << 63);
    flush_column<N>(a, j, xor_sign(1.0, neg), S, B, T);
  }

  // forward permanent: block partials (the reduce kernel sums them in order)
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
    double* p = a.partials + 4 * (size_t)blockIdx.x;
    p[0] = br.hi;
    p[1] = br.lo;
    p[2] = bi.hi;
    p[3] = bi.lo;
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
int launch_grad(const GradArgs& a, int grid, cudaStream_t s);
template <int N>
int grad_blocks_per_sm(int* out);

inline size_t grad_smem_bytes(int N) {
  const int bufs = N >= GRAD_PREFETCH_MIN_N ? 3 : 2;  // suffix products, S (and the prefetched H column)
  return (size_t)N * (N | 1) * sizeof(double2) + (size_t)bufs * N * GRAD_BLOCK * sizeof(double2);
}

}  // namespace permk
