// Row minors of a (K-1) x K matrix in one Gray-code pass, for a batch of items.
//
// For M with rows 0..K-2 and columns 0..K-1, append a free last row x.  The
// Glynn formula (Supp. Eq. (S2)) for the K x K permanent is linear in x:
//   Per([M; x]) = 2^-(K-1) sum_delta (prod delta) (sum_j delta_j x_j) prod_{i<K-1} v_i,
//   v_i = sum_j delta_j M_ij,   delta_0 = +1,
// so the coefficient of x_j, the permanent of M without column j, is
//   m_j = 2^-(K-1) sum_delta (prod delta) delta_j prod_{i<K-1} v_i.
// Per lane: t = (prod delta) prod_i v_i (the forward term over K-1 rows),
// S = running sum of t (registers), H_j = G_j - delta_j S (shared memory, one
// complex per column and lane), which changes only when the Gray code flips
// column j: H_j += 2 delta_j^old S.  At the end G_j = H_j + delta_j S, G_0 = S.
// The per-term cost is that of the forward walk over K-1 rows plus one shared
// read-modify-write.
//
// Element (i, j) of item b is base[b * item_stride + row(i) * rs + col(j) * cs],
// with row(i) = rows ? rows[b * rows_stride + i] : i and col(j) likewise through
// cmap; the boson sampler reads U (transposed: rs = 1, cs = ldu) through the
// drawn output modes and the permuted input modes without gathering a copy.
#pragma once
#include "fwd_kernel.cuh"

namespace permk {

constexpr int MINORS_MAX_K = 32;
constexpr int MINORS_BLOCK = 128;

struct MinorsArgs {
  const double2* base;
  long long rs, cs, item_stride;
  const int* rows;      // nullable
  long long rows_stride;
  const int* cmap;      // nullable
  long long cmap_stride;
  int index_limit;      // row / column indices outside [0, index_limit) read as 0
  const int* status;    // nullable: items with status != 0 are skipped
  int bpi;              // blocks per item
  int chunk_log2;
  uint64_t per_q, per_r;  // floor/ceil split of the 2^(K-1) Gray indices over bpi * block lanes
  double neg_zero;
  double* partials;     // [item][bpi][K][4]: dd (re hi, re lo, im hi, im lo) per column
  int* scale_exp;       // nullable [item]: sum of the row exponents
};

__device__ __forceinline__ int clamp_index(int x, int lim) { return (x >= 0 && x < lim) ? x : 0; }

// R3 (PREC = 3): FP64 row sums and accumulation, the product of the K-1 row sums
// in double-float on the FP32 pipe (as the forward kernel's R3).
// R4 (PREC = 4): double-float row sums and products on the FP32 pipe (as the
// forward kernel's R4), the doubled columns rounded to double-float in shared
// memory and the row sums re-split from FP64 sums of those same columns at every
// chunk start; S and H stay FP64.
template <int K>
__device__ __forceinline__ void minors_walk_df(const double2* Col0, const float4* StepF, double2* Hs, uint64_t kb,
                                               uint64_t ke, uint64_t CH, double& sr, double& si) {
  constexpr int R = K - 1;
  constexpr int NP = Stride<R>::value;
  constexpr int B = MINORS_BLOCK;
  uint64_t k = kb;
  uint64_t g = kb ^ (kb >> 1);
  while (k < ke) {
    const uint64_t c1 = (ke - k > CH) ? k + CH : ke;
    float rh[R], rl[R], ih[R], il[R];
    {
      double vr[R], vi[R];
#pragma unroll
      for (int i = 0; i < R; i++) {
        const double2 x = Col0[i];
        vr[i] = x.x + x.x;
        vi[i] = x.y + x.y;
      }
#pragma unroll 1
      for (int b = 0; b < K - 1; b++) {
        const double coef = ((g >> b) & 1ull) ? -1.0 : 1.0;
        const float4* col = StepF + b * NP;
#pragma unroll
        for (int i = 0; i < R; i++) {
          const float4 x = col[i];
          vr[i] = fma(coef, f32_to_f64_int(x.x) + f32_to_f64_int(x.y), vr[i]);
          vi[i] = fma(coef, f32_to_f64_int(x.z) + f32_to_f64_int(x.w), vi[i]);
        }
      }
#pragma unroll
      for (int i = 0; i < R; i++) {
        const df u = f64_to_df(0.5 * vr[i]), v = f64_to_df(0.5 * vi[i]);
        rh[i] = u.h;
        rl[i] = u.l;
        ih[i] = v.h;
        il[i] = v.l;
      }
    }
#pragma unroll 1
    while (true) {
      df pr, pi;
      prod_dfv<R>(rh, rl, ih, il, pr, pi);
      const double xr = f32_to_f64_int(pr.h) + f32_to_f64_int(pr.l);
      const double xi = f32_to_f64_int(pi.h) + f32_to_f64_int(pi.l);
      const unsigned long long smask = (k & 1ull) << 63;  // prod delta = (-1)^(k & 1)
      sr += xor_sign(xr, smask);
      si += xor_sign(xi, smask);
      ++k;
      if (k >= ke) break;
      const int b = __ffsll((long long)k) - 1;
      {
        const double f = xor_sign(2.0, ((g >> b) & 1ull) << 63);
        double2 h = Hs[(b + 1) * B];
        h.x = fma(f, sr, h.x);
        h.y = fma(f, si, h.y);
        Hs[(b + 1) * B] = h;
      }
      g ^= 1ull << b;
      if (k >= c1) break;
      const float sg = ((g >> b) & 1ull) ? -1.0f : 1.0f;
      const float4* col = StepF + b * NP;
#pragma unroll
      for (int i = 0; i < R; i++) {
        const float4 x = col[i];
        const df u = df_add_signed(df{rh[i], rl[i]}, df{x.x, x.y}, sg);
        const df v = df_add_signed(df{ih[i], il[i]}, df{x.z, x.w}, sg);
        rh[i] = u.h;
        rl[i] = u.l;
        ih[i] = v.h;
        il[i] = v.l;
      }
    }
  }
}

template <int K, int PREC>
__global__ void __launch_bounds__(MINORS_BLOCK, 2) minors_kernel(MinorsArgs a) {
  constexpr int R = K - 1;                      // rows in the product
  constexpr int NP = Stride<(R > 0 ? R : 1)>::value;
  extern __shared__ double2 smem[];
  double2* Col0 = smem;                         // M[:, 0] (scaled rows)
  double2* Step = smem + NP;                    // 2 M[:, b+1], b = 0..K-2
  constexpr int B = MINORS_BLOCK;               // the launch's block size
  double2* Hs = smem + K * NP + threadIdx.x;    // Hs[j * B]: slot 0 holds G_0 at the end
  __shared__ int s_row[R > 0 ? R : 1];
  __shared__ int s_col[K];

  const int item = blockIdx.x / a.bpi;
  const int blk = blockIdx.x - item * a.bpi;
  if (a.status && a.status[item] != 0) {
    // a failed draw: publish zero partials so the consumer reads defined values
    for (int j = threadIdx.x; j < K; j += B) {
      double* p = a.partials + ((size_t)blockIdx.x * K + j) * 4;
      p[0] = p[1] = p[2] = p[3] = 0.0;
    }
    return;
  }

  // ---- stage M: row scaling by 2^{s_i} (s_i from the row's squared norm) ----
  const double2* base = a.base + (long long)item * a.item_stride;
  for (int j = threadIdx.x; j < K; j += B)
    s_col[j] = a.cmap ? clamp_index(a.cmap[(long long)item * a.cmap_stride + j], a.index_limit) : j;
  __syncthreads();
  for (int i = threadIdx.x; i < R; i += B) {
    const int ri = a.rows ? clamp_index(a.rows[(long long)item * a.rows_stride + i], a.index_limit) : i;
    const double2* rowp = base + (long long)ri * a.rs;
    double nrm = 0.0;
    for (int j = 0; j < K; j++) {
      const double2 v = rowp[(long long)s_col[j] * a.cs];
      nrm = fma(v.x, v.x, nrm);
      nrm = fma(v.y, v.y, nrm);
    }
    const int e2 = (int)((__double2hiint(nrm) >> 20) & 0x7FF) - 1023;
    int s = (nrm == 0.0) ? 0 : -(e2 >> 1);
    s = s > 1000 ? 1000 : (s < -1000 ? -1000 : s);
    s_row[i] = s;
    const double f = pow2_double(s);
    for (int j = 0; j < K; j++) {
      const double2 v = rowp[(long long)s_col[j] * a.cs];
      if (j == 0) Col0[i] = make_double2(v.x * f, v.y * f);
      else Step[(j - 1) * NP + i] = make_double2(2.0 * (v.x * f), 2.0 * (v.y * f));
    }
  }
  for (int j = 0; j < K; j++) Hs[j * B] = make_double2(0.0, 0.0);
  __syncthreads();
  if (a.scale_exp && blk == 0 && threadIdx.x == 0) {
    int tot = 0;
    for (int i = 0; i < R; i++) tot += s_row[i];
    a.scale_exp[item] = tot;
  }

  // ---- the lane's Gray range ----
  const uint64_t T = (uint64_t)blk * B + threadIdx.x;
  const uint64_t kb = a.per_q * T + (T < a.per_r ? T : a.per_r);
  const uint64_t ke = kb + a.per_q + (T < a.per_r ? 1 : 0);
  const uint64_t CH = 1ull << a.chunk_log2;
  const double nz = a.neg_zero;
  double sr = 0.0, si = 0.0;  // S
  uint64_t k = kb;
  uint64_t g = kb ^ (kb >> 1);
  if constexpr (PREC == 4 && R >= 2) {
    // the doubled columns to double-float, in place (16 bytes each)
    float4* StepF = reinterpret_cast<float4*>(Step);
    for (int idx = threadIdx.x; idx < (K - 1) * R; idx += B) {
      const int b = idx / R, i = idx % R;
      const double2 v = Step[b * NP + i];
      const df re = f64_to_df(v.x), im = f64_to_df(v.y);
      StepF[b * NP + i] = make_float4(re.h, re.l, im.h, im.l);
    }
    __syncthreads();
    minors_walk_df<K>(Col0, StepF, Hs, kb, ke, CH, sr, si);
    k = ke;
    g = (ke > kb) ? ((ke - 1) ^ ((ke - 1) >> 1)) : g;  // the last term's signs
  } else {
  while (k < ke) {
    const uint64_t c1 = (ke - k > CH) ? k + CH : ke;
    double vr[R > 0 ? R : 1], vi[R > 0 ? R : 1];
    if (R > 0) {
      // exact row sums at the chunk start: (2 M_:0 + sum_b +-2 M_:b+1) / 2
#pragma unroll
      for (int i = 0; i < R; i++) {
        const double2 x = Col0[i];
        vr[i] = x.x + x.x;
        vi[i] = x.y + x.y;
      }
#pragma unroll 1
      for (int b = 0; b < K - 1; b++) {
        const double coef = ((g >> b) & 1ull) ? -1.0 : 1.0;
        const double2* col = Step + b * NP;
#pragma unroll
        for (int i = 0; i < R; i++) {
          const double2 x = col[i];
          vr[i] = fma(coef, x.x, vr[i]);
          vi[i] = fma(coef, x.y, vi[i]);
        }
      }
#pragma unroll
      for (int i = 0; i < R; i++) {
        vr[i] *= 0.5;
        vi[i] *= 0.5;
      }
    }
#pragma unroll 1
    while (true) {
      const unsigned long long smask = (k & 1ull) << 63;  // prod delta = (-1)^(k & 1)
      if constexpr (PREC == 3 && R > 1) {
        // R3: double-float product of the FP64 row sums (FP64 updates and accumulation)
        double pr, pi;
        prod_df<R>(vr, vi, pr, pi);
        sr += xor_sign(pr, smask);
        si += xor_sign(pi, smask);
      } else if (R > 0) {
        term_r0<(R > 0 ? R : 1), 3>(vr, vi, smask, sr, si, nz);
      } else {
        sr += xor_sign(1.0, smask);
      }
      ++k;
      if (k >= ke) break;
      // column b+1 flips: H_{b+1} += 2 delta^old S
      const int b = __ffsll((long long)k) - 1;
      {
        const double f = xor_sign(2.0, ((g >> b) & 1ull) << 63);
        double2 h = Hs[(b + 1) * B];
        h.x = fma(f, sr, h.x);
        h.y = fma(f, si, h.y);
        Hs[(b + 1) * B] = h;
      }
      g ^= 1ull << b;
      if (k >= c1) break;  // next chunk: recompute the row sums from g
      if (R > 0) {
        const double su = xor_sign(1.0, ((g >> b) & 1ull) << 63);
        const double2* col = Step + b * NP;
#pragma unroll
        for (int i = 0; i < R; i++) {
          const double2 x = col[i];
          vr[i] = fma(su, x.x, vr[i]);
          vi[i] = fma(su, x.y, vi[i]);
        }
      }
    }
  }
  }
  // G_j = H_j + delta_j S (delta_0 = +1, H_0 = 0)
  Hs[0] = make_double2(sr, si);
  for (int j = 1; j < K; j++) {
    const double f = xor_sign(1.0, ((g >> (j - 1)) & 1ull) << 63);
    double2 h = Hs[j * B];
    h.x = fma(f, sr, h.x);
    h.y = fma(f, si, h.y);
    Hs[j * B] = h;
  }
  __syncthreads();

  // ---- block sum per column in a fixed order: warp w takes columns w, w + 4, ... ----
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int nwarps = B >> 5;
  const double2* Hb = smem + K * NP;
  for (int j = warp; j < K; j += nwarps) {
    dd tr{0.0, 0.0}, ti{0.0, 0.0};
    for (int t = lane; t < B; t += 32) {
      const double2 v = Hb[j * B + t];
      tr = dd_add(tr, dd{v.x, 0.0});
      ti = dd_add(ti, dd{v.y, 0.0});
    }
    warp_sum_dd(tr, ti);
    if (lane == 0) {
      double* p = a.partials + ((size_t)blockIdx.x * K + j) * 4;
      p[0] = tr.hi;
      p[1] = tr.lo;
      p[2] = ti.hi;
      p[3] = ti.lo;
    }
  }
}

inline size_t minors_smem_bytes(int K) {
  const int R = K - 1;
  const int NP = (R > 0 ? R : 1) | 1;
  return (size_t)K * NP * sizeof(double2) + (size_t)K * MINORS_BLOCK * sizeof(double2);
}

template <int K>
int launch_minors(const MinorsArgs& a, int prec, int grid, cudaStream_t s);
template <int K>
int minors_blocks_per_sm(int prec, int* out);

}  // namespace permk
