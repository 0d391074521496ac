/*
 * perm.h — C ABI of libperm, a GB300 (sm_103a) engine for matrix permanents.
 *
 * The problem (arXiv 1606.05836, Eq. (1) and Supp. "Parallelization and
 * Optimization"): the probability of a boson-sampling outcome is
 *     Pr[S -> T] = |Per(U_ST)|^2 / (s_1! ... s_m! t_1! ... t_m!),
 * and Per(A) of the n x n submatrix is evaluated by Ryser's formula (Supp.
 * Eq. (S1)) or the BB/FG (Glynn) formula (Supp. Eq. (S2)).  The sums are walked
 * in reflected-Gray-code order, so consecutive terms differ by one column.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Matrices are complex128, row-major, a[i][j] = A[i*lda + j], lda >= n, with
 *   perm_c128 layout-compatible with C99 double _Complex / torch.complex128.
 * - Every pointer named d* is DEVICE memory owned by the caller; the library
 *   allocates no device memory.  Entry points that need scratch take a caller
 *   workspace (query its size with the matching *_workspace_size function);
 *   pass a 256-byte-aligned buffer of at least that size (perm_glynn,
 *   perm_ryser, perm_ryser_nw, the range calls and perm_glynn_mult accept
 *   16-byte alignment).  The library never frees it.
 *   (perm_glynn_noalloc instead uses a fixed array compiled into the library.)
 * - Calls are asynchronous and stream-ordered on `stream` (a cudaStream_t;
 *   NULL = the legacy default stream), except prob_sample which synchronises
 *   the stream and returns a host value.  Two calls that share a workspace must
 *   be ordered on one stream.
 * - Host-detectable argument errors return a negative perm_status before
 *   anything is launched; launch failures return PERM_ECUDA.  NaN/Inf entries
 *   propagate to a non-finite result.  Nothing calls exit/abort and no kernel
 *   waits on a flag, so no call can hang the device.
 * - Gray index k in [0, 2^M) addresses one term.  Glynn: M = n-1, delta_1 = +1
 *   and delta_{b+2} = -1 iff bit b of g(k) = k ^ (k >> 1) is set.  Ryser:
 *   M = n, column b+1 is in the subset iff bit b of g(k) is set.
 * - n <= PERM_MAX_N.  n = 0 gives Per = 1.
 */
#ifndef PERM_H_
#define PERM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PERM_MAX_N 48
#define PERM_ABI_VERSION 1

typedef struct {
  double re, im;
} perm_c128;

typedef enum {
  PERM_OK = 0,
  PERM_EINVAL = -1,     /* null pointer, bad lda/stride/option, bad occupation vector */
  PERM_ERANGE = -2,     /* n < 0 or n > PERM_MAX_N, or an index range out of [0, 2^M) */
  PERM_ENOMEM = -3,     /* workspace smaller than required */
  PERM_ECUDA = -4,      /* a CUDA runtime call or launch failed (see perm_last_cuda_error) */
  PERM_ENONFINITE = -5, /* non-finite value where a finite one is required */
  PERM_ETIMEOUT = -6    /* reserved: a bounded wait ran out */
} perm_status;

/* Precision ladder.  FP64 is used in every rung for the row sums recomputed at
 * each chunk start, the accumulation of the terms and the cross-block reduction;
 * R0-R3 also update the row sums in FP64 at every Gray step. */
typedef enum {
  PERM_FP64 = 0,    /* R0: FP64 products, FP64 accumulation of the terms */
  PERM_FP64_DD = 1, /* R1: FP64 products, double-double accumulation of the terms */
  PERM_FP32P_DD = 2, /* R2: FP32 n-way products of the FP64 row sums, double-double accumulation */
  PERM_FP64_DF = 3,  /* R3: the FP64 row sums split into FP32 pairs (~48 bits) and multiplied in
                        double-float arithmetic on the FP32 pipe, FP64 accumulation */
  PERM_FP32X2 = 4    /* R4 (opt-in; relaxes the FP64 row-sum updates the rungs above keep):
                        double-float (FP32 pair, ~48-bit) row sums updated at every step and
                        double-float products, all on the FP32 pipe; exact FP64 row sums at each
                        chunk start (default every 2^10 steps), FP64 accumulation.  Glynn only
                        (perm_glynn, perm_glynn_range, perm_glynn_noalloc, perm_batched with
                        method 0, perm_row_minors, boson_sample); EINVAL elsewhere */
} perm_prec;

/* Launch options; pass NULL for the defaults (every field 0 = default). */
typedef struct {
  int prec;       /* perm_prec */
  int chunk_log2; /* row sums are recomputed from scratch every 2^chunk_log2 steps (default 12; R4: 10; 1..30) */
  int block;      /* threads per block (multiple of 32, 32..256; default 128) */
  int grid;       /* blocks (default: SMs x resident blocks per SM) */
  int unit_log2;  /* perm_batched: Gray indices per lane in one work unit, log2 (default 11, 0..30) */
} perm_opts;

/* --- single permanent ------------------------------------------------------ */

/* Bytes of workspace needed by perm_glynn / perm_ryser / *_range for these
 * options on the current device. */
size_t perm_workspace_size(int n, const perm_opts* opts);

/* Per(A) by the BB/FG (Glynn) formula, Supp. Eq. (S2) and Algorithm 2 of
 * arXiv 1606.05836: all 2^(n-1) delta vectors, then / 2^(n-1).  dOut receives
 * one perm_c128. */
int perm_glynn(const perm_c128* dA, int n, int lda, perm_c128* dOut, void* dWork, size_t workBytes,
               const perm_opts* opts, void* stream);

/* Per(A) by Ryser's formula, Supp. Eq. (S1) and Algorithm 1: the 2^n subsets,
 * then x (-1)^n.  dOut receives one perm_c128. */
int perm_ryser(const perm_c128* dA, int n, int lda, perm_c128* dOut, void* dWork, size_t workBytes,
               const perm_opts* opts, void* stream);

/* Per(A) by Ryser's formula halved to 2^(n-1) subsets (Nijenhuis and Wilf):
 * Per = (-1)^(n-1) 2 sum_{S in [n-1]} (-1)^|S| prod_i (x_i + sum_{j in S} a_ij),
 * x_i = a_{i,n} - (1/2) sum_j a_ij — Eq. (S1) with the same term count as Eq.
 * (S2).  The paper runs only the plain 2^n-subset form; this variant is here for
 * its summation-order and precision comparison.  dOut receives one perm_c128. */
int perm_ryser_nw(const perm_c128* dA, int n, int lda, perm_c128* dOut, void* dWork, size_t workBytes,
                  const perm_opts* opts, void* stream);

/* Partial sums over Gray indices [k_begin, k_end) — the index-range split of
 * Algorithms 1 and 2 (each MPI process took such a range) and the unit a
 * multi-GPU shard computes.  The sum is of the un-normalised signed terms
 * (no 1/2^(n-1), no (-1)^n).  dOut receives two perm_c128: the double-double
 * sum as (hi, lo).  Requires n >= 1 and k_begin <= k_end <= 2^M. */
int perm_glynn_range(const perm_c128* dA, int n, int lda, uint64_t k_begin, uint64_t k_end, perm_c128* dOut,
                     void* dWork, size_t workBytes, const perm_opts* opts, void* stream);
int perm_ryser_range(const perm_c128* dA, int n, int lda, uint64_t k_begin, uint64_t k_end, perm_c128* dOut,
                     void* dWork, size_t workBytes, const perm_opts* opts, void* stream);

/* Per(A) from partial sums over disjoint Gray-index ranges that together cover
 * [0, 2^M): the final reduce of Algorithms 1 and 2 (there an MPI reduce of the
 * per-process sums, followed by the formula's normalisation), for partials
 * computed by perm_glynn_range / perm_ryser_range on several GPUs or boxes, or
 * chunk by chunk in a checkpointed run.
 * hParts: host, [count][2] perm_c128: partial p as the (hi, lo) pair the range
 *         call wrote.  They are added in double-double in the order p = 0 ..
 *         count-1 (pass them in range order for a result that does not depend
 *         on how the work was spread).
 * method: 0 = Glynn (the sum times 2^-(n-1), exact), 1 = Ryser (times (-1)^n).
 * hOut:   host, [2] perm_c128: Per(A) as (hi, lo).
 * Host arithmetic only (no device, no stream).  1 <= n <= PERM_MAX_N,
 * count >= 1; non-finite partials give a non-finite result. */
int perm_combine_partials(const perm_c128* hParts, int count, int n, int method, perm_c128* hOut);

/* --- batched permanents --------------------------------------------------- */

/* Many permanents of mixed sizes 1 <= n_i <= PERM_BATCH_MAX_N in one persistent,
 * size-bucketed launch (largest n first; items cut into work units that warps
 * claim from a shared counter).  This is the batch of output patterns of one
 * interferometer behind Eq. (1) of arXiv 1606.05836.
 *
 * dPacked:  all matrices, row-major, item i at dPacked + dOffsets[i] with lda = n_i.
 * dOffsets: int64 offsets in complex elements (device), dN: int32 sizes (device);
 * hN:       the same sizes on the host (used only to size the workspace layout).
 * method:   0 = Glynn (Eq. (S2)), 1 = Ryser (Eq. (S1)); opts->prec R0-R3 for both,
 *           PERM_FP32X2 (R4) for Glynn only.
 * dScale:   nullable per-item factor for the probability, e.g. 1/(prod s_i! prod t_j!).
 * dOut:     per-item Per (perm_c128).  dProb: nullable per-item |Per|^2 * scale.
 * dWork:    256-byte-aligned workspace of perm_batched_workspace_size() bytes.
 * If dN disagrees with hN so that the plan does not fit, or an n is out of
 * range, the outputs are NaN (no out-of-bounds access).  All kernels are
 * launched on `stream`; the sequence is graph-capturable.  Per item the result
 * is deterministic for fixed options. */
#define PERM_BATCH_MAX_N 32
size_t perm_batched_workspace_size(int count, const int32_t* hN, int method, const perm_opts* opts);
int perm_batched(const perm_c128* dPacked, const int64_t* dOffsets, const int32_t* dN, const int32_t* hN, int count,
                 int method, const double* dScale, perm_c128* dOut, double* dProb, void* dWork, size_t workBytes,
                 const perm_opts* opts, void* stream);

/* --- repeated columns (photon collisions) ------------------------------------ */

/* Per(A) of the n x n matrix whose columns are column c of dB repeated
 * hMult[c] times (c = 0..g-1, sum hMult = n) — the U_ST of Eq. (1) when t_j
 * photons leave output j.  Eq. (S2) with identical columns grouped: a group of m
 * copies enters through k = number of its delta signs that are -1, with
 * binomial weight C(m, k) and row-sum coefficient m - 2k, so the sum has
 * prod over repeated groups (m_c + 1) x 2^(free columns) terms instead of
 * 2^(n-1).  One launch walks the (class, free column) index space: each
 * combination of the repeated groups (a class) is a Gray walk over the free
 * columns, its sum multiplied by the class weight prod C(m_c, k_c) (-1)^k_c.
 * dB: device, row-major n x g, ldb >= g.  hMult: host.  dOut: one perm_c128.
 * Workspace: perm_glynn_mult_workspace_size() bytes, 16-byte aligned.
 * The paper's runs have no repeated columns; this is the collision case Eq. (1)
 * allows (t_j > 1). */
size_t perm_glynn_mult_workspace_size(int n, int g, const int32_t* hMult, const perm_opts* opts);
int perm_glynn_mult(const perm_c128* dB, int n, int ldb, int g, const int32_t* hMult, perm_c128* dOut, void* dWork,
                    size_t workBytes, const perm_opts* opts, void* stream);

/* --- one output probability ------------------------------------------------ */

/* Eq. (1) of arXiv 1606.05836 for one input pattern S and output pattern T:
 *     Pr[S -> T] = |Per(U_ST)|^2 / (s_1! ... s_m! t_1! ... t_m!).
 * dU:  the m x m interferometer unitary (device, row-major, ldu >= m); U[i][j] is
 *      the amplitude from input mode i to output mode j.
 * hS, hT: host occupation vectors of length m with equal sums n <= PERM_MAX_N.
 *      Row r of U_ST is input mode i repeated s_i times (ascending i), column c is
 *      output mode j repeated t_j times (the paper defers U_ST's construction to
 *      Aaronson-Arkhipov; this orientation is the one stated here).
 * hProb: host result.  hPerm: nullable host Per(U_ST).
 * dWork: 256-byte-aligned workspace of prob_sample_workspace_size(n) bytes.
 * U_ST is gathered on the device and Per(U_ST) is the Glynn kernel's; with
 * repeated output (or input) modes the distinct columns (or rows, through the
 * transpose) go through perm_glynn_mult, whichever orientation has fewer terms.
 * The call synchronises `stream` and returns with *hProb written. */
size_t prob_sample_workspace_size(int n, const perm_opts* opts);
int prob_sample(const perm_c128* dU, int m, int ldu, const int32_t* hS, const int32_t* hT, double* hProb,
                perm_c128* hPerm, void* dWork, size_t workBytes, const perm_opts* opts, void* stream);

/* --- adjoint ---------------------------------------------------------------- */

/* Per(A_b) and its derivatives for a batch of matrices, in the same Gray-code
 * pass as the Glynn sum (Supp. Eq. (S2) of arXiv 1606.05836, differentiated:
 * dPer/da_ij = 2^-(n-1) sum_delta (prod delta) delta_j prod_{k != i} v_k; the
 * paper itself has no gradient).  opts->prec PERM_FP64 (default) or PERM_FP64_DF
 * (the prefix, suffix and q products in double-float on the FP32 pipe; row sums,
 * the running sums S, the accumulators H and the flips stay FP64); other values
 * give PERM_EINVAL.  Two adjacent lanes share each Gray walk, half the rows each.
 *
 * dA:        batch matrices, matrix b at dA + b*strideA (complex elements), lda >= n.
 * dPerm:     nullable [batch] Per(A_b).   dAbs2: nullable [batch] |Per(A_b)|^2.
 * dMinor:    nullable [batch][n][n] dPer/da_ij = Per(A_b without row i, column j).
 * dGradAbs2: nullable [batch][n][n] 2 Per conj(dPer/da_ij) = d|Per|^2/dRe a_ij
 *            + i d|Per|^2/dIm a_ij (PyTorch's convention for a real loss).
 * dWork:     256-byte-aligned, perm_grad_workspace_size() bytes: per lane pair one n x n
 *            complex accumulator (grid x 128 pairs x n^2 x 16 bytes, e.g. 0.32 GB at
 *            n = 32).  The batch runs item after item on `stream`.
 * 1 <= n <= PERM_GRAD_MAX_N (n = 0 gives Per = 1, no derivatives). */
#define PERM_GRAD_MAX_N 32
size_t perm_grad_workspace_size(int n, const perm_opts* opts);
int perm_grad(const perm_c128* dA, int n, int lda, int batch, int64_t strideA, perm_c128* dPerm, double* dAbs2,
              perm_c128* dMinor, perm_c128* dGradAbs2, void* dWork, size_t workBytes, const perm_opts* opts,
              void* stream);

/* --- without caller memory ----------------------------------------------- */

/* perm_glynn without a workspace argument: the same computation and kernel as
 * perm_glynn, but the kernel's scratch (the last-block ticket and the per-block
 * partial sums) lives in a fixed array inside the library.  The paper has no
 * counterpart; this exists for callers that cannot allocate device memory —
 * for instance code embedded in a host application that owns and budgets all
 * GPU memory, or a latency-critical path that must not call cudaMalloc because
 * it can synchronise the device and stall other streams.
 *
 * - The array is PERM_NOALLOC_SCRATCH_BYTES of device memory per GPU that loads
 *   the library, held until the process exits; nothing is allocated or freed per
 *   call.  A launch needing more than PERM_NOALLOC_MAX_BLOCKS blocks (an explicit
 *   opts->grid above it) is rejected with PERM_ENOMEM.
 * - The first call on each device looks the array's device address up
 *   (cudaGetSymbolAddress) with that device current; make that first call before
 *   any stream capture begins.  The address is then kept for the life of the
 *   process: after cudaDeviceReset on that device it is stale, so do not call
 *   perm_glynn_noalloc in a process that has reset the device.
 * - All calls share the one array, which keeps the previous call's contents
 *   (the ticket is cleared on the stream before each launch).  Calls whose
 *   kernels overlap on the GPU — different streams or host threads without
 *   ordering between them — race on it: order them on one stream.
 * Arguments and results are as for perm_glynn. */
#define PERM_NOALLOC_MAX_BLOCKS 4096
#define PERM_NOALLOC_SCRATCH_BYTES (256 + 32 * PERM_NOALLOC_MAX_BLOCKS)
int perm_glynn_noalloc(const perm_c128* dA, int n, int lda, perm_c128* dOut, const perm_opts* opts, void* stream);

/* --- row minors and boson-sampling draws ----------------------------------- */

/* The k permanents m_j = Per(M without column j) of (k-1) x k matrices M, in one
 * Gray-code pass per matrix: appending a free last row x to M, Supp. Eq. (S2)
 * of arXiv 1606.05836 is linear in x and m_j is the coefficient of x_j,
 *     m_j = 2^-(k-1) sum_delta (prod delta) delta_j prod_{i<k-1} (sum_l delta_l M_il).
 * (The paper has no such routine; the boson sampler below needs it.)  opts->prec
 * PERM_FP64 (default), PERM_FP64_DF (double-float products of the FP64 row sums)
 * or PERM_FP32X2 (the walk in double-float), as for perm_glynn.
 *
 * dM:    batch matrices (device, complex128, row-major, k-1 rows of k entries,
 *        row stride ldm >= k); matrix b at dM + b*strideM elements.
 * dOut:  [batch][k] device results.
 * dWork: 256-byte-aligned, perm_row_minors_workspace_size(k, batch) bytes
 *        (per block partials: O(batch x blocks per item x k x 32) bytes).
 * 1 <= k <= PERM_MINORS_MAX_K; k = 1 gives m_0 = 1 (the empty permanent).
 * Asynchronous on `stream`; errors as for perm_glynn. */
#define PERM_MINORS_MAX_K 32
size_t perm_row_minors_workspace_size(int k, int batch, const perm_opts* opts);
int perm_row_minors(const perm_c128* dM, int k, int ldm, int batch, int64_t strideM, perm_c128* dOut,
                    void* dWork, size_t workBytes, const perm_opts* opts, void* stream);

/* Draws output patterns of Eq. (1) of arXiv 1606.05836 for n photons in n
 * distinct input modes, by the chain rule of Clifford and Clifford (SODA 2018):
 * the paper only bounds the cost of a draw by that of one permanent.  With
 * A[l][j] = U[in(alpha_j)][l] (U[i][j]: amplitude from input mode i to output
 * mode j, as for prob_sample), step k = 1..n weighs every output mode l by
 *     w_k(l) = |Per(A[(r_1..r_{k-1}, l), (0..k-1)])|^2
 *            = |sum_j A[l][j] Per(A[(r_1..r_{k-1}), (0..k-1) without j])|^2
 * (the k minors by the kernel of perm_row_minors, read straight from U) and
 * takes r_k = the first mode whose running sum of w_k, accumulated in mode order,
 * exceeds u_k * W, W = that sum over all m modes; if rounding leaves u_k W at or
 * above every running sum, the last mode of positive weight.
 *
 * dU:       the m x m unitary (device, row-major, ldu >= m).
 * hInputs:  host, n distinct input modes in [0, m).
 * dAlpha:   device [nsamples][n] int32, each row a permutation of 0..n-1 (the
 *           draw's random photon order), caller-drawn uniformly.
 * dUnif:    device [nsamples][n] doubles in [0, 1) (the draw's uniforms).
 * dR:       device [nsamples][n] int32 out: r_1..r_n (output modes, draw order;
 *           the pattern is their multiset).  A draw whose alpha or uniforms are
 *           invalid, or that meets a step of zero or non-finite total weight,
 *           has all n entries -1.
 * dWork:    256-byte-aligned, boson_sample_workspace_size(m, n, nsamples) bytes
 *           (O(nsamples x (16 m + 8 n) + partials)).
 * opts->prec PERM_FP64 (default), PERM_FP64_DF or PERM_FP32X2 selects the row
 * minors' arithmetic.
 * 1 <= n <= BOSON_SAMPLE_MAX_N, n <= m.  2n - 1 kernel launches, all on
 * `stream`, no host synchronisation (the call may be captured in a CUDA graph
 * once the workspace exists). */
#define BOSON_SAMPLE_MAX_N 32
size_t boson_sample_workspace_size(int m, int n, int nsamples, const perm_opts* opts);
int boson_sample(const perm_c128* dU, int m, int ldu, int n, const int32_t* hInputs, int nsamples,
                 const int32_t* dAlpha, const double* dUnif, int32_t* dR, void* dWork, size_t workBytes,
                 const perm_opts* opts, void* stream);

/* --- diagnostics ----------------------------------------------------------- */

/* FP64 FMA throughput probe: grid x block threads each run
 * PERM_FP64_PROBE_CHAINS independent dependent chains of `iters` fused
 * multiply-adds (x <- x a + b), i.e. grid x block x iters x
 * PERM_FP64_PROBE_CHAINS DFMA instructions, 2 FP64 flops each.  Time it with
 * events on `stream` to measure the FP64 peak against which the permanent
 * kernels' FLOP rates are reported (they are bound by the FP64 pipe).  dSink:
 * one device double that the kernel never actually writes (it keeps the chains
 * live).  iters >= 1, grid >= 1, block a multiple of 32 in 32..1024.
 * Asynchronous. */
#define PERM_FP64_PROBE_CHAINS 4
int perm_fp64_fma_probe(int iters, int grid, int block, double* dSink, void* stream);

const char* perm_strerror(int status);
/* The cudaError_t of the most recent PERM_ECUDA on this host thread (0 if none). */
int perm_last_cuda_error(void);
int perm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PERM_H_ */
