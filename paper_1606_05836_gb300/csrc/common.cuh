// Device helpers shared by the permanent kernels: integer-pipe sign handling,
// double-double sums, FP64<->FP32 conversions on bit patterns, the per-term
// product and the per-thread Gray-code walk.
//
// GB300 FP64 runs at 2 lanes/clk/SM (0.5 per SM sub-partition), ~60x below
// FP32, so everything that is not the method's FP64 arithmetic is moved to the
// integer pipe: term signs and update signs are XORs of sign bits, magnitude
// ordering for compensated sums is an integer compare, and FP64<->FP32
// conversions of the FP32-product rung are done on the bit patterns.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace permk {

// KIND_RYSER_NW: Ryser's formula over the 2^(n-1) subsets of the first n-1
// columns, Per = (-1)^(n-1) 2 sum_S (-1)^|S| prod_i (x_i + sum_{j in S} a_ij),
// x_i = a_{i,n-1} - (1/2) sum_j a_ij (Nijenhuis and Wilf's halving of Eq. (S1)).
// KIND_GLYNN_MULT: Eq. (S2) for a matrix with repeated columns (see MultInfo):
// one class of the multiplicity expansion at a time, v_i = sum_c coef_c b_ic
// over the distinct columns b_c, coef = +-1 for the free (non-repeated)
// columns (-1 iff their bit of g(k) is set), +1 for the fixed singleton, and
// m_c - 2 k_c for a repeated group whose class digit is k_c.
enum { KIND_GLYNN = 0, KIND_RYSER = 1, KIND_RYSER_NW = 2, KIND_GLYNN_MULT = 3 };

// Column structure of a matrix with repeated columns.  Group c (distinct column
// c) is free column role[c] >= 0, the fixed delta = +1 singleton (role -1), or a
// repeated group (role -2) whose class digit k_c = (cls / radix_base[c]) %
// radix[c] counts its -1 signs; radix = m + 1 (m for the group holding the
// fixed copy) and the class weight is prod C(radix_c - 1, k_c) (-1)^k_c.
struct MultInfo {
  int g;
  int nfree;
  signed char role[48];
  unsigned char mult[48];
  unsigned char radix[48];
  long long radix_base[48];
};

__device__ __forceinline__ int mult_digit(const MultInfo& mi, int c, long long cls) {
  return (int)((cls / mi.radix_base[c]) % mi.radix[c]);
}

// prod_c C(radix_c - 1, k_c) (-1)^k_c over the repeated groups (exact: < 2^53)
__device__ inline double mult_class_weight(const MultInfo& mi, long long cls) {
  double w = 1.0;
  int sign = 0;
  for (int c = 0; c < mi.g; c++) {
    if (mi.role[c] != -2) continue;
    const int m = mi.radix[c] - 1, k = mult_digit(mi, c, cls);
    double b = 1.0;
    for (int i = 1; i <= k; i++) b = b * (double)(m - k + i) / (double)i;
    w *= b;
    sign ^= (k & 1);
  }
  return sign ? -w : w;
}

// ---------------------------------------------------------------------------
// small helpers (integer-pipe sign handling, double-double)
// ---------------------------------------------------------------------------

__device__ __forceinline__ double xor_sign(double x, unsigned long long mask) {
  return __longlong_as_double(__double_as_longlong(x) ^ mask);
}

__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// s + x = s' + e exactly (Fast2Sum with the larger magnitude first, chosen by an
// integer compare of the bit patterns); e is accumulated into c.
__device__ __forceinline__ void fast2sum_acc(double& s, double& c, double x) {
  const bool s_big = abs_bits(s) >= abs_bits(x);
  const double big = s_big ? s : x;
  const double small = s_big ? x : s;
  const double t = s + x;
  const double e = small - (t - big);
  c += e;
  s = t;
}

struct dd {
  double hi, lo;
};

__device__ __forceinline__ dd dd_add(dd a, dd b) {
  double s = a.hi + b.hi;
  double bb = s - a.hi;
  double e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  double h = s + e;
  double l = e - (h - s);
  return dd{h, l};
}

// FP64 -> FP32 on the integer pipe: round-half-up of the 52-bit mantissa,
// values below 2^-126 flush to zero, overflow gives infinity.
__device__ __forceinline__ float f64_to_f32_int(double x) {
  const unsigned lo = (unsigned)__double2loint(x);
  const unsigned hi = (unsigned)__double2hiint(x);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu);
  const unsigned mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  unsigned bits = ((unsigned)(e - 896) << 23) + mant + ((lo >> 28) & 1u);
  bits = (e > 896) ? bits : 0u;
  bits = (e < 1151) ? bits : 0x7F800000u;
  return __uint_as_float(sign | bits);
}

// FP32 -> FP64 on the integer pipe (exact for normal numbers; FP32 subnormals -> 0).
__device__ __forceinline__ double f32_to_f64_int(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u;
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned m = u & 0x7FFFFFu;
  unsigned hi = sign | ((e + 896u) << 20) | (m >> 3);
  unsigned lo = m << 29;
  hi = (e == 0u) ? sign : hi;
  lo = (e == 0u) ? 0u : lo;
  hi = (e == 255u) ? (sign | 0x7FF00000u | (m ? 0x80000u : 0u)) : hi;
  lo = (e == 255u) ? 0u : lo;
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ double pow2_double(int s) {
  // 2^s for s in [-1022, 1023]
  return __longlong_as_double((long long)(s + 1023) << 52);
}

// ---------------------------------------------------------------------------
// per-term work
// ---------------------------------------------------------------------------

// TUNE bit 0: Gray update as DFMA(+-1, col, v) instead of DADD with an XOR-ed sign.
// TUNE bit 1: the products' multiplies as DFMA with a -0.0 addend instead of DMUL.
template <int TUNE>
__device__ __forceinline__ double dmul(double x, double y, double nz) {
  if (TUNE & 2) return fma(x, y, nz);
  return x * y;
}

// (pr, pi) <- (pr, pi) * (vr, vi)
template <int TUNE>
__device__ __forceinline__ void cmul_inplace(double& pr, double& pi, double vr, double vi, double nz) {
  const double t = dmul<TUNE>(pi, vi, nz);
  const double u = dmul<TUNE>(pi, vr, nz);
  const double nr = fma(pr, vr, -t);
  const double ni = fma(pr, vi, u);
  pr = nr;
  pi = ni;
}

// R0: acc += sign * prod_i v_i, the last multiply fused into the accumulation.
template <int N, int TUNE>
__device__ __forceinline__ void term_r0(const double (&vr)[N], const double (&vi)[N], unsigned long long smask,
                                        double& ar, double& ai, double nz) {
  if (N == 1) {
    ar += xor_sign(vr[0], smask);
    ai += xor_sign(vi[0], smask);
    return;
  }
  double pr = vr[0], pi = vi[0];
#pragma unroll
  for (int i = 1; i < N - 1; i++) cmul_inplace<TUNE>(pr, pi, vr[i], vi[i], nz);
  pr = xor_sign(pr, smask);
  pi = xor_sign(pi, smask);
  ar = fma(pr, vr[N - 1], ar);
  ar = fma(-pi, vi[N - 1], ar);
  ai = fma(pr, vi[N - 1], ai);
  ai = fma(pi, vr[N - 1], ai);
}

// full FP64 product (R1)
template <int N, int TUNE>
__device__ __forceinline__ void prod_f64(const double (&vr)[N], const double (&vi)[N], double& pr, double& pi,
                                         double nz) {
  pr = vr[0];
  pi = vi[0];
#pragma unroll
  for (int i = 1; i < N; i++) cmul_inplace<TUNE>(pr, pi, vr[i], vi[i], nz);
}

// FP32 product of the FP64 row sums (R2); conversions on the integer pipe.
template <int N>
__device__ __forceinline__ void prod_f32(const double (&vr)[N], const double (&vi)[N], double& pr, double& pi) {
  float qr = f64_to_f32_int(vr[0]);
  float qi = f64_to_f32_int(vi[0]);
#pragma unroll
  for (int i = 1; i < N; i++) {
    const float xr = f64_to_f32_int(vr[i]);
    const float xi = f64_to_f32_int(vi[i]);
    const float nr = fmaf(qr, xr, -qi * xi);
    const float ni = fmaf(qr, xi, qi * xr);
    qr = nr;
    qi = ni;
  }
  pr = f32_to_f64_int(qr);
  pi = f32_to_f64_int(qi);
}

// ---------------------------------------------------------------------------
// R3: double-float products (pairs of FP32 on the FP32 pipe)
// ---------------------------------------------------------------------------

struct df {
  float h, l;
};

// Exact split of an FP64 value into hi + lo FP32 halves on the integer pipe:
// hi = the 53-bit mantissa rounded to 24 bits, lo = the rounded residual (24 of
// its <= 29 bits), so hi + lo carries ~48 bits.  |x| < 2^-126 flushes hi to 0
// and |x| < 2^-74 flushes lo to 0 (rows are pre-scaled to norm ~1).
__device__ __forceinline__ df f64_to_df(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  const int e = (int)((u >> 52) & 0x7FFull);
  const long long m = (long long)((u & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
  const long long H = (m + (1ll << 28)) >> 29;
  const long long R = m - (H << 29);
  unsigned hb = ((unsigned)(e - 897) << 23) + (unsigned)H;
  hb = (e > 896) ? hb : 0u;
  hb = (e < 1151) ? hb : 0x7F800000u;
  const int le = e - 948;  // biased FP32 exponent of 2^(e - 1075), the residual's unit
  const float unit = __uint_as_float((le > 0 && le < 255) ? ((unsigned)le << 23) : 0u);
  const float lo = __fmul_rn(__int2float_rn((int)R), unit);
  return df{__uint_as_float(sign | hb), __uint_as_float(__float_as_uint(lo) ^ sign)};
}

// (xr + i xi) <- (xr + i xi)(yr + i yi) in double-float: exact products of the
// high parts (two-product by FMA), a two-sum of the two, the cross terms with the
// low parts folded in by FMA, then renormalisation.  The _rn intrinsics keep the
// compiler from contracting the error-free transformations.
__device__ __forceinline__ void dfc_mul(df& xr, df& xi, const df yr, const df yi) {
  const float p1 = __fmul_rn(xr.h, yr.h), e1 = __fmaf_rn(xr.h, yr.h, -p1);
  const float p2 = __fmul_rn(xi.h, yi.h), e2 = __fmaf_rn(xi.h, yi.h, -p2);
  const float s = __fsub_rn(p1, p2);
  const float bb = __fsub_rn(s, p1);
  const float es = __fadd_rn(__fsub_rn(p1, __fsub_rn(s, bb)), __fsub_rn(-p2, bb));
  float t = __fadd_rn(es, __fsub_rn(e1, e2));
  t = __fmaf_rn(xr.h, yr.l, t);
  t = __fmaf_rn(xr.l, yr.h, t);
  t = __fmaf_rn(-xi.h, yi.l, t);
  t = __fmaf_rn(-xi.l, yi.h, t);
  const float rh = __fadd_rn(s, t);
  const float rl = __fsub_rn(t, __fsub_rn(rh, s));
  const float q1 = __fmul_rn(xr.h, yi.h), f1 = __fmaf_rn(xr.h, yi.h, -q1);
  const float q2 = __fmul_rn(xi.h, yr.h), f2 = __fmaf_rn(xi.h, yr.h, -q2);
  const float u = __fadd_rn(q1, q2);
  const float cc = __fsub_rn(u, q1);
  const float eu = __fadd_rn(__fsub_rn(q1, __fsub_rn(u, cc)), __fsub_rn(q2, cc));
  float v = __fadd_rn(eu, __fadd_rn(f1, f2));
  v = __fmaf_rn(xr.h, yi.l, v);
  v = __fmaf_rn(xr.l, yi.h, v);
  v = __fmaf_rn(xi.h, yr.l, v);
  v = __fmaf_rn(xi.l, yr.h, v);
  const float ih = __fadd_rn(u, v);
  const float il = __fsub_rn(v, __fsub_rn(ih, u));
  xr = df{rh, rl};
  xi = df{ih, il};
}

// prod_i v_i in double-float, returned as FP64 (hi + lo is exact in FP64)
template <int N>
__device__ __forceinline__ void prod_df(const double (&vr)[N], const double (&vi)[N], double& pr, double& pi) {
  df ar = f64_to_df(vr[0]), ai = f64_to_df(vi[0]);
#pragma unroll
  for (int i = 1; i < N; i++) dfc_mul(ar, ai, f64_to_df(vr[i]), f64_to_df(vi[i]));
  pr = f32_to_f64_int(ar.h) + f32_to_f64_int(ar.l);
  pi = f32_to_f64_int(ai.h) + f32_to_f64_int(ai.l);
}

// R4: double-float row sums as well, so the whole walk runs on the FP32 pipe.

// prod_i v_i of double-float values (one chain of n - 1 multiplies).
template <int N>
__device__ __forceinline__ void prod_dfv(const float (&rh)[N], const float (&rl)[N], const float (&ih)[N],
                                         const float (&il)[N], df& pr, df& pi) {
  pr = df{rh[0], rl[0]};
  pi = df{ih[0], il[0]};
#pragma unroll
  for (int i = 1; i < N; i++) dfc_mul(pr, pi, df{rh[i], rl[i]}, df{ih[i], il[i]});
}

// a + sg * b in double-float for sg = +-1: Dekker's double-length addition (two-
// sum of the high parts, low parts added, renormalised) with the sign folded into
// the FMAs (sg * b is exact, so each FMA rounds exactly as the plain sum would);
// the _rn intrinsics keep the error-free steps from being contracted.
__device__ __forceinline__ df df_add_signed(const df a, const df b, float sg) {
  const float s = __fmaf_rn(sg, b.h, a.h);
  const float bb = __fsub_rn(s, a.h);
  const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fmaf_rn(sg, b.h, -bb));
  const float t = __fadd_rn(e, __fmaf_rn(sg, b.l, a.l));
  const float h = __fadd_rn(s, t);
  return df{h, __fsub_rn(t, __fsub_rn(h, s))};
}

// Glynn walk over [kb, ke) with double-float row sums: exact FP64 row sums at
// every chunk start (from Acol), split into double-float; each step adds or
// subtracts the flipped doubled column (StepF, double-float (re h, re l, im h,
// im l)); the double-float product goes to FP64 exactly and is accumulated in FP64.
template <int N>
__device__ __forceinline__ void walk_range_df(const double2* __restrict__ Acol, const float4* __restrict__ StepF,
                                              int stride, uint64_t kb, uint64_t ke, uint64_t CH, double& ar,
                                              double& ai) {
  for (uint64_t c0 = kb; c0 < ke;) {
    const uint64_t c1 = (ke - c0 > CH) ? c0 + CH : ke;
    uint64_t g = c0 ^ (c0 >> 1);
    float rh[N], rl[N], ih[N], il[N];
    {
      double vr[N], vi[N];
#pragma unroll
      for (int i = 0; i < N; i++) {
        vr[i] = 0.0;
        vi[i] = 0.0;
      }
#pragma unroll 1
      for (int j = 0; j < N; j++) {
        const double coef = (j == 0) ? 1.0 : (((g >> (j - 1)) & 1ull) ? -1.0 : 1.0);
        const double2* col = Acol + j * stride;
#pragma unroll
        for (int i = 0; i < N; i++) {
          const double2 x = col[i];
          vr[i] = fma(coef, x.x, vr[i]);
          vi[i] = fma(coef, x.y, vi[i]);
        }
      }
#pragma unroll
      for (int i = 0; i < N; i++) {
        const df a = f64_to_df(vr[i]), b = f64_to_df(vi[i]);
        rh[i] = a.h;
        rl[i] = a.l;
        ih[i] = b.h;
        il[i] = b.l;
      }
    }
    uint64_t k = c0;
#pragma unroll 1
    while (true) {
      df pr, pi;
      prod_dfv<N>(rh, rl, ih, il, pr, pi);
      // to FP64 exactly (hi + lo fits), converted on the integer pipe: hardware
      // conversions measured slower here (FP64-pipe dispatch stalls)
      const double xr = f32_to_f64_int(pr.h) + f32_to_f64_int(pr.l);
      const double xi = f32_to_f64_int(pi.h) + f32_to_f64_int(pi.l);
      const unsigned long long smask = (k & 1ull) << 63;  // (prod delta) = (-1)^(k & 1)
      ar += xor_sign(xr, smask);
      ai += xor_sign(xi, smask);
      ++k;
      if (k >= c1) break;
      const int b = __ffsll((long long)k) - 1;
      g ^= 1ull << b;
      // bit now set: delta_{b+2} became -1, subtract 2a; bit now clear: add
      const float sg = ((g >> b) & 1ull) ? -1.0f : 1.0f;
      const float4* col = StepF + b * stride;
#pragma unroll
      for (int i = 0; i < N; i++) {
        const float4 x = col[i];
        const df u = df_add_signed(df{rh[i], rl[i]}, df{x.x, x.y}, sg);
        const df v = df_add_signed(df{ih[i], il[i]}, df{x.z, x.w}, sg);
        rh[i] = u.h;
        rl[i] = u.l;
        ih[i] = v.h;
        il[i] = v.l;
      }
    }
    c0 = c1;
  }
}

// ---------------------------------------------------------------------------
// one thread's Gray walk over [kb, ke) (steps a2-a5)
// ---------------------------------------------------------------------------

template <bool GLOBAL>
__device__ __forceinline__ double2 ldcol(const double2* p) {
  if (GLOBAL) return __ldg(p);
  return *p;
}

// Walks Gray indices [kb, ke): at every chunk start (every CH steps from kb) the
// row sums are recomputed exactly from the columns Acol (v_i = base_i + sum_j
// coef_j a_ij; Glynn: base 0, coef_0 = +1 and coef_{b+1} = -1 iff bit b of g(k)
// is set; Ryser: base 0, coef_b = [bit b of g(k)]; Ryser-NW: base x_i (the
// vector Xb), coef_b = [bit b] over the first n-1 columns); every other step
// adds +-Step[b], b = ctz(k).  Columns are `stride` complex numbers apart.
// GLOBAL selects read-only global loads instead of shared-memory loads.
// Per-thread (sum, compensation) -> normalised double-double.
template <int PREC>
__device__ __forceinline__ void acc_to_dd(double ar, double ai, double cr, double ci, dd& sr, dd& si) {
  if (PREC == 1 || PREC == 2) {
    sr = dd_add(dd{ar, 0.0}, dd{cr, 0.0});
    si = dd_add(dd{ai, 0.0}, dd{ci, 0.0});
  } else {
    sr = dd{ar, 0.0};
    si = dd{ai, 0.0};
  }
}

// KIND_GLYNN_MULT: Acol holds the g distinct columns, Step the doubled free
// columns (by free index) and mi the column structure; [kb, ke) are indices
// K = class * 2^nfree + free-column Gray index.  A class boundary ends a chunk
// (so no lane walks a second segment alone), and each chunk's sum is added to
// (tot_r, tot_i) times its class weight.
template <int N, int PREC, int TUNE, bool GLOBAL>
__device__ __forceinline__ void walk_range(const double2* __restrict__ Acol, const double2* __restrict__ Step,
                                           const double2* __restrict__ Xb, const MultInfo* mi, dd* tot_r,
                                           dd* tot_i, int stride, int kind, uint64_t kb, uint64_t ke, uint64_t CH,
                                           double nz, double& ar, double& ai, double& cr, double& ci) {
  const bool glynn = (kind == KIND_GLYNN);
  const bool multk = (kind == KIND_GLYNN_MULT);
  const bool glynn_signs = glynn || multk;
  const bool has_base = (kind == KIND_RYSER_NW);
  // Glynn: a set Gray bit means delta = -1 (subtract 2a when it turns on);
  // Ryser: a set bit means the column is in S (add a when it turns on).
  const unsigned long long on_mask = glynn_signs ? 0x8000000000000000ull : 0ull;
  const int ncols = (kind == KIND_RYSER_NW) ? N - 1 : (multk ? mi->g : N);
  // index within a class of the repeated-column expansion (the whole index otherwise)
  const uint64_t lmask = multk ? ((1ull << mi->nfree) - 1ull) : ~0ull;
  for (uint64_t c0 = kb; c0 < ke;) {
    uint64_t c1 = (ke - c0 > CH) ? c0 + CH : ke;
    long long cls = 0;
    if (multk) {
      cls = (long long)(c0 >> mi->nfree);
      const uint64_t bnd = ((uint64_t)cls + 1) << mi->nfree;
      if (c1 > bnd) c1 = bnd;
      ar = ai = cr = ci = 0.0;  // this chunk's sum, weighted below
    }
    const uint64_t gidx = c0 & lmask;
    uint64_t g = gidx ^ (gidx >> 1);
    double vr[N], vi[N];
    // exact row sums at the chunk start: v_i = base_i + sum_j coef_j a_ij
    if (has_base) {
#pragma unroll
      for (int i = 0; i < N; i++) {
        const double2 x = ldcol<GLOBAL>(Xb + i);
        vr[i] = x.x;
        vi[i] = x.y;
      }
    } else {
#pragma unroll
      for (int i = 0; i < N; i++) {
        vr[i] = 0.0;
        vi[i] = 0.0;
      }
    }
#pragma unroll 1
    for (int j = 0; j < ncols; j++) {
      double coef;
      if (glynn) {
        coef = (j == 0) ? 1.0 : (((g >> (j - 1)) & 1ull) ? -1.0 : 1.0);
      } else if (multk) {
        const int role = mi->role[j];
        if (role >= 0) coef = ((g >> role) & 1ull) ? -1.0 : 1.0;
        else if (role == -1) coef = 1.0;
        else coef = (double)(mi->mult[j] - 2 * mult_digit(*mi, j, cls));
      } else {
        coef = ((g >> j) & 1ull) ? 1.0 : 0.0;
      }
      const double2* col = Acol + j * stride;
#pragma unroll
      for (int i = 0; i < N; i++) {
        const double2 x = ldcol<GLOBAL>(col + i);
        vr[i] = fma(coef, x.x, vr[i]);
        vi[i] = fma(coef, x.y, vi[i]);
      }
    }
    uint64_t k = c0;
#pragma unroll 1
    while (true) {
      // term sign (prod delta) = (-1)^popcount(g) = (-1)^(index & 1)
      const unsigned long long smask = ((k & lmask) & 1ull) << 63;
      if (PREC == 0) {
        term_r0<N, TUNE>(vr, vi, smask, ar, ai, nz);
      } else if (PREC == 3) {
        double pr, pi;
        prod_df<N>(vr, vi, pr, pi);
        ar += xor_sign(pr, smask);
        ai += xor_sign(pi, smask);
      } else {
        double pr, pi;
        if (PREC == 1) prod_f64<N, TUNE>(vr, vi, pr, pi, nz);
        else prod_f32<N>(vr, vi, pr, pi);
        fast2sum_acc(ar, cr, xor_sign(pr, smask));
        fast2sum_acc(ai, ci, xor_sign(pi, smask));
      }
      ++k;
      if (k >= c1) break;
      // Gray step: bit b = ctz(k) flips (k is not a class start inside a chunk)
      const int b = __ffsll((long long)k) - 1;
      g ^= 1ull << b;
      // negative iff (Glynn and the bit turned on) or (Ryser and it turned off)
      const unsigned long long umask = ((((g >> b) & 1ull) ^ 1ull) << 63) ^ on_mask;
      const double2* col = Step + b * stride;
      if (TUNE & 1) {
        const double sgn = xor_sign(1.0, umask);
#pragma unroll
        for (int i = 0; i < N; i++) {
          const double2 x = ldcol<GLOBAL>(col + i);
          vr[i] = fma(sgn, x.x, vr[i]);
          vi[i] = fma(sgn, x.y, vi[i]);
        }
      } else {
#pragma unroll
        for (int i = 0; i < N; i++) {
          const double2 x = ldcol<GLOBAL>(col + i);
          vr[i] += xor_sign(x.x, umask);
          vi[i] += xor_sign(x.y, umask);
        }
      }
    }
    if (multk) {
      // the chunk lies in one class: add its sum times the class weight
      dd pr, pi;
      acc_to_dd<PREC>(ar, ai, cr, ci, pr, pi);
      const double w = mult_class_weight(*mi, cls);
      *tot_r = dd_add(*tot_r, dd{pr.hi * w, pr.lo * w});
      *tot_i = dd_add(*tot_i, dd{pi.hi * w, pi.lo * w});
    }
    c0 = c1;
  }
}

// Warp butterfly sum of double-double pairs (every lane ends with the same sum).
__device__ __forceinline__ void warp_sum_dd(dd& sr, dd& si) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    dd orr{__shfl_xor_sync(0xffffffffu, sr.hi, off), __shfl_xor_sync(0xffffffffu, sr.lo, off)};
    dd oii{__shfl_xor_sync(0xffffffffu, si.hi, off), __shfl_xor_sync(0xffffffffu, si.lo, off)};
    sr = dd_add(sr, orr);
    si = dd_add(si, oii);
  }
}


}  // namespace permk
