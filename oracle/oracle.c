/*
 * CPU oracle for the matrix permanent — TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * leg may load this library.  It shares no code, header or table with the CUDA
 * path in paper_1606_05836_gb300/csrc and must never be called by it.
 *
 * Plain, slow, obviously-correct evaluations of what the GPU path computes
 * (arXiv 1606.05836, "A Benchmark Test of Boson Sampling on Tianhe-2"):
 *
 *   oracle_perm_def      Per(A) = sum over permutations s of prod_i a[i][s(i)]
 *                        (the definition; the paper names the permanent but never
 *                        writes it out), complex _Float128, depth-first over s.
 *   oracle_ryser_range   partial sums of Ryser's formula, Supp. Eq. (S1), with the
 *                        subset S of each iteration taken from the bits of the
 *                        iteration index (Algorithm 1) or of its reflected Gray
 *                        code; the row sums of every subset are recomputed from
 *                        scratch, as Algorithm 1 does; complex _Float128.
 *   oracle_glynn_range   partial sums of the BB/FG (Glynn) formula, Supp. Eq. (S2),
 *                        delta_1 = +1 and delta_{b+2} = -1 iff bit b of the index
 *                        (or of its Gray code) is set; complex _Float128.
 *   oracle_glynn_gray    Eq. (S2) summed in reflected-Gray-code order, the
 *                        execution order the paper names as the O(n 2^n)
 *                        alternative (Supp. "Parallelization and Optimization"):
 *                        consecutive delta vectors differ in one sign, so each
 *                        row sum changes by +-2 a_ij; complex _Float128 with the
 *                        row sums recomputed from scratch at every thread's start.
 *   oracle_glynn_f64dd_range / oracle_ryser_f64dd_range / oracle_glynn_f64dd
 *                        Eq. (S2) / Eq. (S1) in reflected-Gray order in IEEE
 *                        FP64 (row sums, their one-sign updates and the n-way
 *                        products), each term added to a double-double
 *                        accumulator (Knuth's TwoSum); the index range is cut
 *                        into pieces of 2^6 consecutive indices, each started
 *                        from row sums computed from scratch (the per-process
 *                        split of Algorithms 1 and 2 with more, smaller
 *                        pieces).  Fast enough for n = 29-40 on a many-core host.
 *   oracle_ryser_z128    Eq. (S1) for integer matrices in unsigned __int128
 *                        arithmetic (exact modulo 2^128, hence exact whenever
 *                        |Per(A)| < 2^127).
 *   oracle_minors        Per of every (n-1)x(n-1) minor, i.e. dPer/da_ij by the
 *                        Laplace expansion, each by oracle_ryser_range.
 *   oracle_prob          Eq. (1): |Per(U_ST)|^2 / (prod s_i! prod t_j!).
 *
 * Matrices are row-major, n x n, complex entries interleaved as (re, im)
 * doubles: a[i][j] = (A[2(i*n+j)], A[2(i*n+j)+1]).  Results are returned as
 * (re_hi, re_lo, im_hi, im_lo) doubles, hi + lo being the _Float128 result
 * rounded to about 106 bits.
 *
 * Work over an index range is split into contiguous per-thread pieces as the
 * paper's Algorithms 1 and 2 split it across processes (OpenMP here); each piece
 * sums in index order and the pieces are added in thread order.
 *
 * Parity pins: every function is pinned by tests/test_oracle_pins.py (closed
 * forms from the paper's precision tables, derangement numbers, brute-force
 * matching counts, diagonal / rank-one / block-diagonal products, Laplace
 * expansion, invariances, sum of probabilities = 1).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef _Float128 q_t;
typedef struct { q_t re, im; } qc_t;

static inline qc_t qc_add(qc_t a, qc_t b) { qc_t r = {a.re + b.re, a.im + b.im}; return r; }
static inline qc_t qc_sub(qc_t a, qc_t b) { qc_t r = {a.re - b.re, a.im - b.im}; return r; }
static inline qc_t qc_mul(qc_t a, qc_t b) {
  qc_t r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
  return r;
}
static inline qc_t qc_zero(void) { qc_t r = {0, 0}; return r; }
static inline qc_t qc_one(void) { qc_t r = {1, 0}; return r; }

static inline qc_t load_entry(const double* A, int n, int i, int j) {
  qc_t r = {(q_t)A[2 * (i * n + j)], (q_t)A[2 * (i * n + j) + 1]};
  return r;
}

static void store_result(qc_t v, double* out4) {
  double rh = (double)v.re, ih = (double)v.im;
  out4[0] = rh;
  out4[1] = (double)(v.re - (q_t)rh);
  out4[2] = ih;
  out4[3] = (double)(v.im - (q_t)ih);
}

static int max_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
  nthreads = 1;
#endif
  return nthreads < 1 ? 1 : nthreads;
}

/* ------------------------------------------------------------------ */
/* Definition: sum over all permutations (depth-first).                */
/* ------------------------------------------------------------------ */

static qc_t perm_dfs(const double* A, int n, int row, uint64_t used, qc_t prefix) {
  if (row == n) return prefix;
  qc_t total = qc_zero();
  for (int col = 0; col < n; col++) {
    if (used & (1ull << col)) continue;
    qc_t next = qc_mul(prefix, load_entry(A, n, row, col));
    total = qc_add(total, perm_dfs(A, n, row + 1, used | (1ull << col), next));
  }
  return total;
}

/* Per(A) from its definition.  n <= 11 (n! leaves).  Returns 0 or -1 (bad n). */
int oracle_perm_def(int n, const double* A, double* out4) {
  if (n < 0 || n > 11 || (n > 0 && !A) || !out4) return -1;
  store_result(perm_dfs(A, n, 0, 0, qc_one()), out4);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Ryser, Supp. Eq. (S1)                                               */
/* ------------------------------------------------------------------ */

static inline uint64_t code_of(uint64_t k, int gray) { return gray ? (k ^ (k >> 1)) : k; }

static inline int popcount64(uint64_t x) { return __builtin_popcountll(x); }

/* One Ryser term: (-1)^{|S|} prod_i sum_{j in S} a_ij, S = bits of `set`. */
static qc_t ryser_term(const double* A, int n, uint64_t set) {
  qc_t prod = qc_one();
  for (int i = 0; i < n; i++) {
    qc_t rowsum = qc_zero();
    for (int j = 0; j < n; j++)
      if (set & (1ull << j)) rowsum = qc_add(rowsum, load_entry(A, n, i, j));
    prod = qc_mul(prod, rowsum);
  }
  if (popcount64(set) & 1) prod = qc_sub(qc_zero(), prod);
  return prod;
}

/* Partial Ryser sum over iteration indices k in [k_begin, k_end), the subset of
 * index k being the bits of k (gray = 0, Algorithm 1) or of k ^ (k >> 1)
 * (gray = 1).  No (-1)^n factor.  Requires 1 <= n <= 48, k_end <= 2^n. */
int oracle_ryser_range(int n, const double* A, uint64_t k_begin, uint64_t k_end, int gray,
                       int nthreads, double* out4) {
  if (n < 1 || n > 48 || !A || !out4) return -1;
  if (k_begin > k_end || k_end > (1ull << n)) return -1;
  int P = max_threads(nthreads);
  uint64_t total = k_end - k_begin;
  qc_t* part = (qc_t*)calloc((size_t)P, sizeof(qc_t));
  if (!part) return -1;
#pragma omp parallel num_threads(P)
  {
#ifdef _OPENMP
    int rank = omp_get_thread_num();
    int np = omp_get_num_threads();
#else
    int rank = 0, np = 1;
#endif
    uint64_t len = (total + (uint64_t)np - 1) / (uint64_t)np;
    uint64_t start = k_begin + (uint64_t)rank * len;
    uint64_t end = start + len;
    if (start > k_end) start = k_end;
    if (end > k_end) end = k_end;
    qc_t acc = qc_zero();
    for (uint64_t k = start; k < end; k++) acc = qc_add(acc, ryser_term(A, n, code_of(k, gray)));
    part[rank] = acc;
  }
  qc_t sum = qc_zero();
  for (int r = 0; r < P; r++) sum = qc_add(sum, part[r]);
  free(part);
  store_result(sum, out4);
  return 0;
}

static qc_t ryser_full_q(const double* A, int n, int nthreads) {
  double r4[4];
  if (n == 0) return qc_one();
  oracle_ryser_range(n, A, 1, 1ull << n, 0, nthreads, r4);
  qc_t s = {(q_t)r4[0] + (q_t)r4[1], (q_t)r4[2] + (q_t)r4[3]};
  if (n & 1) s = qc_sub(qc_zero(), s);
  return s;
}

/* Per(A) by Eq. (S1): (-1)^n sum over non-empty subsets.  n <= 30. */
int oracle_ryser(int n, const double* A, int nthreads, double* out4) {
  if (n < 0 || n > 30 || (n > 0 && !A) || !out4) return -1;
  store_result(ryser_full_q(A, n, nthreads), out4);
  return 0;
}

/* ------------------------------------------------------------------ */
/* BB/FG (Glynn), Supp. Eq. (S2)                                       */
/* ------------------------------------------------------------------ */

/* One Glynn term: (prod_k delta_k) prod_i sum_j delta_j a_ij with delta_1 = +1
 * and delta_{b+2} = -1 iff bit b of `code` is set. */
static qc_t glynn_term(const double* A, int n, uint64_t code) {
  qc_t prod = qc_one();
  for (int i = 0; i < n; i++) {
    qc_t rowsum = qc_zero();
    for (int j = 0; j < n; j++) {
      int negative = (j > 0) && ((code >> (j - 1)) & 1);
      qc_t a = load_entry(A, n, i, j);
      rowsum = negative ? qc_sub(rowsum, a) : qc_add(rowsum, a);
    }
    prod = qc_mul(prod, rowsum);
  }
  if (popcount64(code) & 1) prod = qc_sub(qc_zero(), prod);
  return prod;
}

/* Partial Glynn sum over k in [k_begin, k_end) (no 1/2^{n-1} factor).
 * Requires 1 <= n <= 48, k_end <= 2^{n-1}. */
int oracle_glynn_range(int n, const double* A, uint64_t k_begin, uint64_t k_end, int gray,
                       int nthreads, double* out4) {
  if (n < 1 || n > 48 || !A || !out4) return -1;
  if (k_begin > k_end || k_end > (1ull << (n - 1))) return -1;
  int P = max_threads(nthreads);
  uint64_t total = k_end - k_begin;
  qc_t* part = (qc_t*)calloc((size_t)P, sizeof(qc_t));
  if (!part) return -1;
#pragma omp parallel num_threads(P)
  {
#ifdef _OPENMP
    int rank = omp_get_thread_num();
    int np = omp_get_num_threads();
#else
    int rank = 0, np = 1;
#endif
    uint64_t len = (total + (uint64_t)np - 1) / (uint64_t)np;
    uint64_t start = k_begin + (uint64_t)rank * len;
    uint64_t end = start + len;
    if (start > k_end) start = k_end;
    if (end > k_end) end = k_end;
    qc_t acc = qc_zero();
    for (uint64_t k = start; k < end; k++) acc = qc_add(acc, glynn_term(A, n, code_of(k, gray)));
    part[rank] = acc;
  }
  qc_t sum = qc_zero();
  for (int r = 0; r < P; r++) sum = qc_add(sum, part[r]);
  free(part);
  store_result(sum, out4);
  return 0;
}

/* Per(A) by Eq. (S2): sum over the 2^{n-1} delta vectors, divided by 2^{n-1}. */
int oracle_glynn(int n, const double* A, int nthreads, double* out4) {
  if (n < 0 || n > 30 || (n > 0 && !A) || !out4) return -1;
  if (n == 0) { store_result(qc_one(), out4); return 0; }
  double r4[4];
  oracle_glynn_range(n, A, 0, 1ull << (n - 1), 0, nthreads, r4);
  q_t scale = (q_t)1;
  for (int i = 0; i < n - 1; i++) scale = scale / (q_t)2;
  qc_t s = {((q_t)r4[0] + (q_t)r4[1]) * scale, ((q_t)r4[2] + (q_t)r4[3]) * scale};
  store_result(s, out4);
  return 0;
}

/* Per(A) by Eq. (S2) with the 2^{n-1} delta vectors taken in reflected-Gray order
 * k = 0, 1, ..., delta_{b+2} = -1 iff bit b of k ^ (k >> 1) is set.  Each thread
 * takes a contiguous range of k, computes the row sums of its first delta from
 * scratch, then moves to the next delta by flipping the one sign that changes
 * (row sums change by -+2 a_{i,b+1}).  Complex _Float128.  n <= 40. */
int oracle_glynn_gray(int n, const double* A, int nthreads, double* out4) {
  if (n < 0 || n > 40 || (n > 0 && !A) || !out4) return -1;
  if (n == 0) { store_result(qc_one(), out4); return 0; }
  const uint64_t total = 1ull << (n - 1);
  int P = max_threads(nthreads);
  qc_t* part = (qc_t*)calloc((size_t)P, sizeof(qc_t));
  if (!part) return -1;
  int fail = 0;
#pragma omp parallel num_threads(P)
  {
#ifdef _OPENMP
    int rank = omp_get_thread_num();
    int np = omp_get_num_threads();
#else
    int rank = 0, np = 1;
#endif
    uint64_t len = (total + (uint64_t)np - 1) / (uint64_t)np;
    uint64_t start = (uint64_t)rank * len;
    uint64_t end = start + len;
    if (start > total) start = total;
    if (end > total) end = total;
    qc_t* v = (qc_t*)malloc(sizeof(qc_t) * (size_t)n);
    qc_t acc = qc_zero();
    if (!v) {
#pragma omp atomic write
      fail = 1;
    } else if (start < end) {
      uint64_t code = start ^ (start >> 1);
      for (int i = 0; i < n; i++) {  /* row sums of the first delta, from scratch */
        v[i] = qc_zero();
        for (int j = 0; j < n; j++) {
          int negative = (j > 0) && ((code >> (j - 1)) & 1);
          v[i] = negative ? qc_sub(v[i], load_entry(A, n, i, j)) : qc_add(v[i], load_entry(A, n, i, j));
        }
      }
      for (uint64_t k = start; k < end; k++) {
        qc_t prod = qc_one();
        for (int i = 0; i < n; i++) prod = qc_mul(prod, v[i]);
        acc = (popcount64(code) & 1) ? qc_sub(acc, prod) : qc_add(acc, prod);
        if (k + 1 == end) break;
        int b = __builtin_ctzll(k + 1);   /* the one sign that changes */
        code ^= 1ull << b;
        int now_negative = (code >> b) & 1;
        for (int i = 0; i < n; i++) {
          qc_t a2 = load_entry(A, n, i, b + 1);
          a2.re = a2.re + a2.re;
          a2.im = a2.im + a2.im;
          v[i] = now_negative ? qc_sub(v[i], a2) : qc_add(v[i], a2);
        }
      }
    }
    free(v);
    part[rank] = acc;
  }
  qc_t sum = qc_zero();
  for (int r = 0; r < P; r++) sum = qc_add(sum, part[r]);
  free(part);
  if (fail) return -1;
  q_t scale = (q_t)1;
  for (int i = 0; i < n - 1; i++) scale = scale / (q_t)2;
  sum.re *= scale;
  sum.im *= scale;
  store_result(sum, out4);
  return 0;
}

/* ------------------------------------------------------------------ */
/* FP64 Gray-order sums with double-double accumulation                */
/* ------------------------------------------------------------------ */

/* A double-double number hi + lo, |lo| <= ulp(hi) / 2. */
typedef struct { double hi, lo; } dd_t;

/* hi + lo = a + b exactly (Knuth's TwoSum, no ordering of a and b needed). */
static inline dd_t two_sum(double a, double b) {
  dd_t r;
  r.hi = a + b;
  double bv = r.hi - a;
  r.lo = (a - (r.hi - bv)) + (b - bv);
  return r;
}

/* (a.hi + a.lo) + x rounded to double-double. */
static inline dd_t dd_add_double(dd_t a, double x) {
  dd_t s = two_sum(a.hi, x);
  return two_sum(s.hi, s.lo + a.lo);
}

/* (a.hi + a.lo) + (b.hi + b.lo) rounded to double-double. */
static inline dd_t dd_add_dd(dd_t a, dd_t b) {
  dd_t s = two_sum(a.hi, b.hi);
  return two_sum(s.hi, s.lo + (a.lo + b.lo));
}

#define F64DD_PIECE_LOG2 6

/* Sum over the Gray indices k in [k_begin, k_end) of
 *   Glynn (glynn = 1): (prod_k delta_k) prod_i sum_j delta_j a_ij, delta_1 = +1 and
 *                      delta_{b+2} = -1 iff bit b of g(k) = k ^ (k >> 1) is set;
 *   Ryser (glynn = 0): (-1)^{|S|} prod_i sum_{j in S} a_ij, column b in S iff bit b
 *                      of g(k) is set,
 * in FP64 with the terms accumulated in double-double.  The range is cut at the
 * multiples of 2^F64DD_PIECE_LOG2; every piece computes its first row sums from
 * scratch (in column order) and then follows the Gray code, one column per step.
 * Threads take contiguous runs of pieces; the thread sums are added in thread
 * order.  out4 = (re_hi, re_lo, im_hi, im_lo). */
static int f64dd_gray_sum(int n, const double* A, int glynn, uint64_t k_begin, uint64_t k_end, int nthreads,
                          double* out4) {
  const uint64_t L = 1ull << F64DD_PIECE_LOG2;
  const uint64_t p_first = k_begin / L;
  const uint64_t p_count = (k_end > k_begin) ? (k_end - 1) / L - p_first + 1 : 0;
  int P = max_threads(nthreads);
  dd_t* part = (dd_t*)calloc(2 * (size_t)P, sizeof(dd_t));
  if (!part) return -1;
  int fail = 0;
#pragma omp parallel num_threads(P)
  {
#ifdef _OPENMP
    int rank = omp_get_thread_num();
    int np = omp_get_num_threads();
#else
    int rank = 0, np = 1;
#endif
    uint64_t q = p_count / (uint64_t)np, r = p_count % (uint64_t)np;
    uint64_t pb = p_first + (uint64_t)rank * q + ((uint64_t)rank < r ? (uint64_t)rank : r);
    uint64_t pe = pb + q + ((uint64_t)rank < r ? 1 : 0);
    double* vr = (double*)malloc(sizeof(double) * (size_t)n);
    double* vi = (double*)malloc(sizeof(double) * (size_t)n);
    dd_t acc_re = {0.0, 0.0}, acc_im = {0.0, 0.0};
    if (!vr || !vi) {
#pragma omp atomic write
      fail = 1;
    } else {
      for (uint64_t p = pb; p < pe; p++) {
        uint64_t start = p * L > k_begin ? p * L : k_begin;
        uint64_t end = (p + 1) * L < k_end ? (p + 1) * L : k_end;
        uint64_t code = start ^ (start >> 1);
        for (int i = 0; i < n; i++) {  /* row sums of the piece's first index, from scratch */
          vr[i] = 0.0;
          vi[i] = 0.0;
          for (int j = 0; j < n; j++) {
            const double ar = A[2 * (i * n + j)], ai = A[2 * (i * n + j) + 1];
            if (glynn) {
              int negative = (j > 0) && ((code >> (j - 1)) & 1);
              vr[i] = negative ? vr[i] - ar : vr[i] + ar;
              vi[i] = negative ? vi[i] - ai : vi[i] + ai;
            } else if ((code >> j) & 1) {
              vr[i] += ar;
              vi[i] += ai;
            }
          }
        }
        for (uint64_t k = start; k < end; k++) {
          double pr = vr[0], pi = vi[0];
          for (int i = 1; i < n; i++) {
            double nr = pr * vr[i] - pi * vi[i];
            double ni = pr * vi[i] + pi * vr[i];
            pr = nr;
            pi = ni;
          }
          if (popcount64(code) & 1) {
            pr = -pr;
            pi = -pi;
          }
          acc_re = dd_add_double(acc_re, pr);
          acc_im = dd_add_double(acc_im, pi);
          if (k + 1 == end) break;
          int b = __builtin_ctzll(k + 1); /* the one bit of g that changes */
          code ^= 1ull << b;
          int now_set = (code >> b) & 1;
          if (glynn) {
            /* delta_{b+2} turned to -1 (bit set): subtract 2 a; back to +1: add 2 a */
            for (int i = 0; i < n; i++) {
              const double ar = A[2 * (i * n + b + 1)], ai = A[2 * (i * n + b + 1) + 1];
              vr[i] = now_set ? vr[i] - (ar + ar) : vr[i] + (ar + ar);
              vi[i] = now_set ? vi[i] - (ai + ai) : vi[i] + (ai + ai);
            }
          } else {
            /* column b entered S (bit set): add it; left S: subtract it */
            for (int i = 0; i < n; i++) {
              const double ar = A[2 * (i * n + b)], ai = A[2 * (i * n + b) + 1];
              vr[i] = now_set ? vr[i] + ar : vr[i] - ar;
              vi[i] = now_set ? vi[i] + ai : vi[i] - ai;
            }
          }
        }
      }
    }
    free(vr);
    free(vi);
    part[2 * rank] = acc_re;
    part[2 * rank + 1] = acc_im;
  }
  dd_t sre = {0.0, 0.0}, sim = {0.0, 0.0};
  for (int r = 0; r < P; r++) {
    sre = dd_add_dd(sre, part[2 * r]);
    sim = dd_add_dd(sim, part[2 * r + 1]);
  }
  free(part);
  if (fail) return -1;
  out4[0] = sre.hi;
  out4[1] = sre.lo;
  out4[2] = sim.hi;
  out4[3] = sim.lo;
  return 0;
}

/* Un-normalised Glynn partial sum over Gray indices [k_begin, k_end), FP64 terms,
 * double-double sum.  1 <= n <= 48, k_end <= 2^{n-1}. */
int oracle_glynn_f64dd_range(int n, const double* A, uint64_t k_begin, uint64_t k_end, int nthreads,
                             double* out4) {
  if (n < 1 || n > 48 || !A || !out4) return -1;
  if (k_begin > k_end || k_end > (1ull << (n - 1))) return -1;
  return f64dd_gray_sum(n, A, 1, k_begin, k_end, nthreads, out4);
}

/* Un-normalised Ryser partial sum over Gray indices [k_begin, k_end) (no (-1)^n),
 * FP64 terms, double-double sum.  1 <= n <= 48, k_end <= 2^n. */
int oracle_ryser_f64dd_range(int n, const double* A, uint64_t k_begin, uint64_t k_end, int nthreads,
                             double* out4) {
  if (n < 1 || n > 48 || !A || !out4) return -1;
  if (k_begin > k_end || k_end > (1ull << n)) return -1;
  return f64dd_gray_sum(n, A, 0, k_begin, k_end, nthreads, out4);
}

/* Per(A) by Eq. (S2): the FP64 Gray-order sum over all 2^{n-1} delta vectors
 * (double-double accumulation) times 2^{-(n-1)} (exact).  n <= 48. */
int oracle_glynn_f64dd(int n, const double* A, int nthreads, double* out4) {
  if (n < 0 || n > 48 || (n > 0 && !A) || !out4) return -1;
  if (n == 0) {
    out4[0] = 1.0; out4[1] = 0.0; out4[2] = 0.0; out4[3] = 0.0;
    return 0;
  }
  int rc = f64dd_gray_sum(n, A, 1, 0, 1ull << (n - 1), nthreads, out4);
  if (rc) return rc;
  for (int c = 0; c < 4; c++) out4[c] = ldexp(out4[c], -(n - 1));
  return 0;
}

/* ------------------------------------------------------------------ */
/* Exact integer Ryser (mod 2^128)                                     */
/* ------------------------------------------------------------------ */

/* Per(A) of an integer matrix by Eq. (S1) in unsigned __int128 (two's
 * complement wrap-around).  Exact whenever |Per(A)| < 2^127.  A is row-major
 * int64, n x n.  out2 = (low 64 bits, high 64 bits).  n <= 40. */
int oracle_ryser_z128(int n, const int64_t* A, int nthreads, uint64_t* out2) {
  if (n < 0 || n > 40 || (n > 0 && !A) || !out2) return -1;
  typedef unsigned __int128 u128;
  if (n == 0) { out2[0] = 1; out2[1] = 0; return 0; }
  int P = max_threads(nthreads);
  u128* part = (u128*)calloc((size_t)P, sizeof(u128));
  if (!part) return -1;
  uint64_t k_end = 1ull << n;
#pragma omp parallel num_threads(P)
  {
#ifdef _OPENMP
    int rank = omp_get_thread_num();
    int np = omp_get_num_threads();
#else
    int rank = 0, np = 1;
#endif
    uint64_t total = k_end - 1;
    uint64_t len = (total + (uint64_t)np - 1) / (uint64_t)np;
    uint64_t start = 1 + (uint64_t)rank * len;
    uint64_t end = start + len;
    if (start > k_end) start = k_end;
    if (end > k_end) end = k_end;
    u128 acc = 0;
    for (uint64_t set = start; set < end; set++) {
      u128 prod = 1;
      for (int i = 0; i < n; i++) {
        u128 rowsum = 0;
        for (int j = 0; j < n; j++)
          if (set & (1ull << j)) rowsum += (u128)(__int128)A[i * n + j];
        prod *= rowsum;
      }
      if (popcount64(set) & 1) acc -= prod; else acc += prod;
    }
    part[rank] = acc;
  }
  u128 sum = 0;
  for (int r = 0; r < P; r++) sum += part[r];
  free(part);
  if (n & 1) sum = (u128)0 - sum;
  out2[0] = (uint64_t)sum;
  out2[1] = (uint64_t)(sum >> 64);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Minors: dPer/da_ij = Per(A without row i and column j)             */
/* ------------------------------------------------------------------ */

/* out is n*n*4 doubles: entry (i, j) at out[4*(i*n+j)].  2 <= n <= 24. */
int oracle_minors(int n, const double* A, int nthreads, double* out) {
  if (n < 2 || n > 24 || !A || !out) return -1;
  int m = n - 1;
  int P = max_threads(nthreads);
  int fail = 0;
#pragma omp parallel for num_threads(P) schedule(dynamic, 1)
  for (int ij = 0; ij < n * n; ij++) {
    int i = ij / n, j = ij % n;
    double* M = (double*)malloc(sizeof(double) * 2 * (size_t)m * (size_t)m);
    if (!M) { fail = 1; continue; }
    for (int r = 0, rr = 0; r < n; r++) {
      if (r == i) continue;
      for (int c = 0, cc = 0; c < n; c++) {
        if (c == j) continue;
        M[2 * (rr * m + cc)] = A[2 * (r * n + c)];
        M[2 * (rr * m + cc) + 1] = A[2 * (r * n + c) + 1];
        cc++;
      }
      rr++;
    }
    store_result(ryser_full_q(M, m, 1), out + 4 * (size_t)ij);
    free(M);
  }
  return fail ? -1 : 0;
}

/* ------------------------------------------------------------------ */
/* Eq. (1): output probability                                         */
/* ------------------------------------------------------------------ */

/* U is m x m (row-major interleaved complex); U[i][j] is the amplitude from
 * input mode i to output mode j.  s and t are occupation vectors of length m with
 * equal sums n <= 26.  U_ST has row r = input mode i repeated s_i times
 * (ascending i) and column c = output mode j repeated t_j times.
 * out2 = (probability hi, lo); perm4 (nullable) = Per(U_ST). */
int oracle_prob(int m, const double* U, const int32_t* s, const int32_t* t, int nthreads,
                double* out2, double* perm4) {
  if (m < 1 || !U || !s || !t || !out2) return -1;
  int n = 0, nt = 0;
  for (int i = 0; i < m; i++) {
    if (s[i] < 0 || t[i] < 0) return -1;
    n += s[i];
    nt += t[i];
  }
  if (n != nt || n > 26) return -1;
  int* rows = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  int* cols = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  double* M = (double*)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n * n : 1));
  if (!rows || !cols || !M) { free(rows); free(cols); free(M); return -1; }
  int r = 0, c = 0;
  for (int i = 0; i < m; i++) for (int k = 0; k < s[i]; k++) rows[r++] = i;
  for (int j = 0; j < m; j++) for (int k = 0; k < t[j]; k++) cols[c++] = j;
  for (int a = 0; a < n; a++)
    for (int b = 0; b < n; b++) {
      M[2 * (a * n + b)] = U[2 * (rows[a] * m + cols[b])];
      M[2 * (a * n + b) + 1] = U[2 * (rows[a] * m + cols[b]) + 1];
    }
  qc_t per = ryser_full_q(M, n, nthreads);
  q_t denom = 1;
  for (int i = 0; i < m; i++) {
    for (int k = 2; k <= s[i]; k++) denom *= (q_t)k;
    for (int k = 2; k <= t[i]; k++) denom *= (q_t)k;
  }
  q_t pr = (per.re * per.re + per.im * per.im) / denom;
  out2[0] = (double)pr;
  out2[1] = (double)(pr - (q_t)out2[0]);
  if (perm4) store_result(per, perm4);
  free(rows); free(cols); free(M);
  return 0;
}

int oracle_abi_version(void) { return 1; }
