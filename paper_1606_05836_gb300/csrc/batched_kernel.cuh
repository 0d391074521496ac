// Batched permanents of mixed sizes in one persistent, size-bucketed launch.
//
// Pipeline (all on the device, so the whole sequence can be captured in one
// CUDA graph):
//   0. batch_mult_kernel   per item (Glynn, R0-R2): finds bitwise-identical
//                          columns (photon collisions, t_j > 1 in Eq. (1)); an
//                          item with repeated columns walks the multiplicity
//                          expansion of Eq. (S2) (prod (m_c + 1) x 2^free terms
//                          instead of 2^(n-1), as perm_glynn_mult does).
//   1. batch_plan_kernel   one block: validates n, buckets the items by n
//                          (largest first), cuts every item's index range into
//                          work units of 32 lanes x 2^l terms and prefix-sums the
//                          unit counts and the per-item column storage.
//   2. batch_prep_kernel   per item: rows scaled by powers of two, columns
//                          stored contiguously (column-major), and for Glynn the
//                          doubled step columns (for an item with repeated
//                          columns: its distinct columns and the doubled free
//                          ones).
//   3. batch_walk_kernel   persistent: each warp claims the next unit with one
//                          atomicAdd (bounded by the unit count, no waiting),
//                          runs the same per-lane Gray walk as the single
//                          permanent kernel (dispatching on n), and writes the
//                          unit's double-double partial sum.
//   4. batch_reduce_kernel per item: its units' partials in unit order
//                          (deterministic), scaling, and the probability
//                          epilogue |Per|^2 * scale (Eq. (1) with scale =
//                          1/(prod s_i! prod t_j!)).
#pragma once
#include "common.cuh"

namespace permk {

constexpr int BATCH_MAX_N = 32;
constexpr int BATCH_PLAN_THREADS = 1024;

__host__ __device__ inline int batch_M(int n, int kind) { return kind == KIND_GLYNN ? n - 1 : n; }

// ceil(log2(terms)) for terms >= 1
__host__ __device__ inline int batch_ceil_log2(long long terms) {
  int c = 0;
  while ((1ll << c) < terms) c++;
  return c;
}

// log2 of the indices per lane in one work unit of an item with `terms` indices
// (2^M for a plain item, classes x 2^free with repeated columns)
__host__ __device__ inline int batch_lane_log2(long long terms, int unit_log2) {
  int l = batch_ceil_log2(terms) - 5;
  if (l < 0) l = 0;
  if (l > unit_log2) l = unit_log2;
  return l;
}

// Work units of an item.  With repeated columns the count never exceeds the
// plain item's (fewer terms at the same or a smaller unit), so workspaces sized
// from 2^M hold every plan.
__host__ __device__ inline long long batch_units(long long terms, int unit_log2) {
  const long long per_unit = 32ll << batch_lane_log2(terms, unit_log2);
  return (terms + per_unit - 1) / per_unit;
}

__host__ __device__ inline long long batch_prep_elems(int n, int kind) {
  return (long long)n * n * (kind == KIND_GLYNN ? 2 : 1);
}

struct BatchArgs {
  const double2* packed;   // all matrices, row-major, item i at packed + offsets[i], lda = n_i
  const long long* offsets;
  const int* ns;
  int count;
  int kind;
  int prec;                // R4: the doubled step columns are stored as double-float
  int unit_log2;
  int chunk_log2;
  double neg_zero;
  // workspace
  unsigned long long* cursor;
  int* status;
  long long* total_units;
  int* order;            // sorted position -> item
  int* pos;              // item -> sorted position
  long long* unit_start; // [count + 1], by sorted position
  long long* prep_off;   // [count], by item
  int* scale_exp;        // [count]
  double* partials;      // 4 doubles per unit
  long long* terms;      // [count]: index-space size of each item (set by batch_mult_kernel)
  MultInfo* mult;        // [count]: column structure; g = 0 for an item without repeated columns
  signed char* mcol;     // [count][BATCH_MAX_N]: original column of distinct column c
  int use_mult;          // Glynn R0-R2: walk items with repeated columns by the multiplicity expansion
  double2* prep;
  long long units_cap;
  long long prep_cap;
  // outputs
  const double* scale;   // nullable
  double2* out;
  double* prob;          // nullable
};

enum { BATCH_OK = 0, BATCH_BAD_N = 1, BATCH_NO_ROOM = 2 };

// One lane's walk over [kb, ke) of an item of size n: the plain Gray walk, or
// (mi != nullptr, rungs R0-R2) the multiplicity expansion, whose class-weighted
// chunk sums go to (tr, ti).
template <int PREC, int TUNE>
__device__ __forceinline__ void batch_walk_n(int n, const double2* Acol, const double2* Step, bool glynn,
                                             const MultInfo* mi, dd* tr, dd* ti, uint64_t kb, uint64_t ke, uint64_t CH,
                                             double nz, double& ar, double& ai, double& cr, double& ci) {
  switch (n) {
#define PERM_BCASE(N)                                                                                      \
  case N:                                                                                                  \
    if constexpr (PREC == 4) {                                                                             \
      walk_range_df<N>(Acol, reinterpret_cast<const float4*>(Step), N, kb, ke, CH, ar, ai);                \
    } else if constexpr (PREC == 3) {                                                                      \
      walk_range<N, PREC, TUNE, true>(Acol, Step, nullptr, nullptr, nullptr, nullptr, N,                   \
                                      glynn ? KIND_GLYNN : KIND_RYSER, kb, ke, CH, nz, ar, ai, cr, ci);     \
    } else {                                                                                               \
      if (mi != nullptr)                                                                                   \
        walk_range<N, PREC, TUNE, true>(Acol, Step, nullptr, mi, tr, ti, N, KIND_GLYNN_MULT, kb, ke, CH,   \
                                        nz, ar, ai, cr, ci);                                                \
      else                                                                                                 \
        walk_range<N, PREC, TUNE, true>(Acol, Step, nullptr, nullptr, nullptr, nullptr, N,                 \
                                        glynn ? KIND_GLYNN : KIND_RYSER, kb, ke, CH, nz, ar, ai, cr, ci);   \
    }                                                                                                      \
    break;
    PERM_BCASE(1) PERM_BCASE(2) PERM_BCASE(3) PERM_BCASE(4) PERM_BCASE(5) PERM_BCASE(6) PERM_BCASE(7)
    PERM_BCASE(8) PERM_BCASE(9) PERM_BCASE(10) PERM_BCASE(11) PERM_BCASE(12) PERM_BCASE(13) PERM_BCASE(14)
    PERM_BCASE(15) PERM_BCASE(16) PERM_BCASE(17) PERM_BCASE(18) PERM_BCASE(19) PERM_BCASE(20) PERM_BCASE(21)
    PERM_BCASE(22) PERM_BCASE(23) PERM_BCASE(24) PERM_BCASE(25) PERM_BCASE(26) PERM_BCASE(27) PERM_BCASE(28)
    PERM_BCASE(29) PERM_BCASE(30) PERM_BCASE(31) PERM_BCASE(32)
#undef PERM_BCASE
    default:
      break;
  }
}

template <int PREC, int TUNE>
__global__ void __launch_bounds__(256, 1) batch_walk_kernel(BatchArgs a) {
  if (*a.status != BATCH_OK) return;
  const int lane = threadIdx.x & 31;
  const long long total = *a.total_units;
  const uint64_t CH = 1ull << a.chunk_log2;
  const bool glynn = (a.kind == KIND_GLYNN);
  const double nz = a.neg_zero;
  for (;;) {
    long long u = 0;
    if (lane == 0) u = (long long)atomicAdd(a.cursor, 1ull);
    u = __shfl_sync(0xffffffffu, u, 0);
    if (u >= total) break;
    int lo = 0, hi = a.count - 1;  // largest sorted position with unit_start <= u
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.unit_start[mid] <= u) lo = mid;
      else hi = mid - 1;
    }
    const int item = a.order[lo];
    const int n = a.ns[item];
    const uint64_t terms = (uint64_t)a.terms[item];
    const int ll = batch_lane_log2((long long)terms, a.unit_log2);
    const long long j = u - a.unit_start[lo];
    const uint64_t k0 = ((uint64_t)j * 32ull + (uint64_t)lane) << ll;
    const uint64_t kb = k0 < terms ? k0 : terms;
    const uint64_t ke = (k0 + (1ull << ll)) < terms ? k0 + (1ull << ll) : terms;
    const double2* Acol = a.prep + a.prep_off[item];
    const double2* Step = glynn ? Acol + n * n : Acol;
    const MultInfo* mi = (a.use_mult && a.mult[item].g > 0) ? a.mult + item : nullptr;
    double ar = 0.0, ai = 0.0, cr = 0.0, ci = 0.0;
    dd sr{0.0, 0.0}, si{0.0, 0.0};
    batch_walk_n<PREC, TUNE>(n, Acol, Step, glynn, mi, &sr, &si, kb, ke, CH, nz, ar, ai, cr, ci);
    if (mi == nullptr) acc_to_dd<PREC>(ar, ai, cr, ci, sr, si);
    warp_sum_dd(sr, si);
    if (lane == 0) {
      double* p = a.partials + 4 * (size_t)u;
      p[0] = sr.hi;
      p[1] = sr.lo;
      p[2] = si.hi;
      p[3] = si.lo;
    }
  }
}

template <int PREC>
int launch_batch_walk(const BatchArgs& a, int grid, int block, cudaStream_t s);
template <int PREC>
int batch_walk_blocks_per_sm(int block, int* out);

}  // namespace permk
