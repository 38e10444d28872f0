/*
 * ttgb.h - C ABI of the GB300 TT-rounding library.
 *
 * Implements the hot path of Coulaud, Giraud & Iannacito, "On some
 * orthogonalization schemes in Tensor Train format": TT sums, TT dot
 * products, TT-rounding and the six TT orthogonalization schemes
 * (Algorithms 1-8), on one GPU, in hand-written CUDA for sm_103a.
 *
 * TT format (Section 2): x = x_1 x_2 ... x_d with cores
 * x_k in R^{r_{k-1} x n_k x r_k}, r_0 = r_d = 1.  A core is stored on the
 * device row-major as [r_{k-1}][n_k][r_k] (r_k fastest), so its left
 * unfolding (r_{k-1} n_k) x r_k and its right unfolding r_{k-1} x (n_k r_k)
 * are both contiguous row-major matrices.
 *
 * Conventions shared by every entry point:
 *  - All calls are ordered on the context's CUDA stream.  Calls that return
 *    a host scalar (tt_dot, tt_norm, tt_round's ranks, ...) synchronize that
 *    stream before returning.
 *  - Inputs are never modified.  Every tt_tensor** output is allocated by the
 *    library and released with tt_tensor_free.  On error no output is
 *    produced: *out is set to NULL and nothing has to be freed.
 *  - Errors: a NULL pointer, d < 1, m < 1, delta < 0 or NaN, r_0 != 1,
 *    r_d != 1 or a rank < 1 give TT_ERR_ARG; differing orders or mode sizes
 *    give TT_ERR_SHAPE; an allocation beyond the context's HBM budget (or a
 *    failed device allocation) gives TT_ERR_OOM; a failed CUDA call gives
 *    TT_ERR_CUDA (the message is kept, see tt_last_error).
 *  - The library is not thread-safe per context; distinct contexts may be
 *    used from distinct threads.
 */
#ifndef TTGB_H
#define TTGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TT_OK = 0,
    TT_ERR_ARG = 1,        /* invalid argument */
    TT_ERR_SHAPE = 2,      /* orders or mode sizes differ */
    TT_ERR_OOM = 3,        /* HBM budget exceeded or device allocation failed */
    TT_ERR_NOT_SPD = 4,    /* TT-Gram: Cholesky of the Gram matrix failed */
    TT_ERR_BREAKDOWN = 5,  /* zero vector where a scheme normalises */
    TT_ERR_NONFINITE = 6,  /* NaN or Inf met in a result */
    TT_ERR_TIMEOUT = 7,    /* a bounded device wait ran out, or a server wait timed out */
    TT_ERR_CUDA = 8,       /* a CUDA runtime call failed */
    TT_ERR_CANCELLED = 9   /* a served request was cancelled before it started */
} tt_status;

/* Arithmetic of a context.
 * TT_FP64:       cores, GEMMs, Cholesky, SVD and norms in FP64.
 * TT_MIXED_TF32: cores stored in FP32; the first pass's Gram matrix of every
 *                Cholesky QR (and the second pass's for unfoldings of length
 *                >= 4096) on tcgen05 tensor cores in TF32 with FP32
 *                accumulation; the GEMMs that produce core values (apply
 *                Q = L^{-1} X, absorb core L) on CUDA cores in FP32 by
 *                default (the split-TF32 tensor-core GEMM of tt_gemm_f32 is
 *                opt-in: environment variable TTGB_TC_GEMM=3 or 2 when the
 *                context is created); small r x r factorizations in FP32;
 *                norm, thresholds and tail sums in FP64; truncation SVDs in
 *                FP64 (FP32 column Jacobi with an FP64-measured residual
 *                guard for ranks >= 32).
 * TT_FP32:       cores and every GEMM in FP32 on CUDA cores (no tensor
 *                cores); small factorizations as TT_MIXED_TF32. */
typedef enum { TT_FP64 = 0, TT_MIXED_TF32 = 1, TT_FP32 = 2 } tt_precision;

/* Algorithms 1-5 and 8. */
typedef enum {
    TT_CGS = 0, TT_MGS = 1, TT_CGS2 = 2, TT_MGS2 = 3, TT_GRAM = 4, TT_HOUSEHOLDER = 5
} tt_scheme;

/* TT_ROUND_PAPER rounds where Algorithms 1-5 and 8 round.
 * TT_ROUND_EVERY_UPDATE also rounds the running vector after every axpy of
 * the projection loops (for Householder: every reflected a_j); a loop that
 * makes no update keeps the single rounding of the paper policy. */
typedef enum { TT_ROUND_PAPER = 0, TT_ROUND_EVERY_UPDATE = 1 } tt_round_policy;

/* Householder sign rule for r(i) in TTH-vec (Algorithm 6).
 * TT_SIGN_STABLE: r(i) = -sign(<a, f_i>) sqrt(||a||^2 - s), the
 * cancellation-free choice of Section 3.3 (default).
 * TT_SIGN_LITERAL: r(i) = +sign(<a, f_i>) sqrt(...), as printed in the
 * listing.  sign(0) = +1 in both. */
typedef enum { TT_SIGN_STABLE = 0, TT_SIGN_LITERAL = 1 } tt_sign_rule;

/* Storage type of a tensor's cores. */
typedef enum { TT_DTYPE_F64 = 0, TT_DTYPE_F32 = 1 } tt_dtype;

typedef struct tt_ctx tt_ctx;        /* stream, workspace, HBM budget, stats */
typedef struct tt_tensor tt_tensor;  /* d, n[], r[], device cores */

/* Counters of a context (reset by tt_ctx_reset_stats). */
typedef struct {
    uint64_t kernel_launches;  /* kernels this library launched */
    uint64_t roundings;        /* tt_round calls, including those inside schemes */
    uint64_t host_syncs;       /* stream synchronizations made */
    uint64_t bytes_in_use;     /* device bytes held by live tensors + workspace */
    uint64_t peak_bytes;       /* high-water mark of bytes_in_use */
    uint64_t svd_calls;        /* truncation SVDs actually computed */
    uint64_t certified_bonds;  /* bonds kept whole by the sigma_min certificate */
    uint64_t fallback_orth;    /* orthogonalizations that took the shifted path */
    uint64_t svd_sweeps;       /* Jacobi sweeps of the truncation SVDs (counted
                                  only while profiling is on: it costs a sync) */
    uint64_t series_passes;    /* second Cholesky QR passes replaced by the
                                  series (I + E)^(-1/2) of a near-identity Gram */
    uint64_t series_retries;   /* roundings redone with Cholesky passes because a
                                  series pass met a Gram too far from I */
    uint64_t second_pass_skips; /* certified left-to-right bonds whose first
                                   Cholesky QR pass was already orthonormal to
                                   the required level (second pass not run) */
    uint64_t fallback_fp32;    /* fallback orthogonalizations of FP32 data kept
                                  in FP32 (exactly rank-deficient unfoldings);
                                  the rest of fallback_orth ran in FP64 */
} tt_stats;

/* Per-kernel timing of a context (tt_ctx_set_profiling): CUDA events are
 * recorded on the context's stream around every instrumented launch. */
typedef struct {
    char name[32];       /* kernel family, e.g. "gram_tf32_tc", "gemm_f32" */
    uint64_t launches;
    double total_ms;     /* sum of event-measured durations */
    double flops;        /* algorithmic floating-point operations */
    double bytes;        /* algorithmic HBM bytes (operands read + result written) */
} tt_kernel_profile;

/* ---- context ---------------------------------------------------------- */

/* Creates a context on CUDA device `device`.  `cuda_stream` is a
 * cudaStream_t owned by the caller (NULL = the legacy default stream).
 * `hbm_budget` caps the device bytes the context may hold (0 = no cap);
 * a call that would exceed it fails with TT_ERR_OOM before touching the GPU.
 * Returns TT_ERR_CUDA if the device is absent or not sm_103. */
tt_status tt_ctx_create(tt_ctx** ctx, int device, tt_precision prec,
                        void* cuda_stream, size_t hbm_budget);
/* Releases the caller's reference.  Tensors still alive keep the context
 * (and their memory) valid until they are freed; the context must not be
 * used for new calls after tt_ctx_destroy. */
void      tt_ctx_destroy(tt_ctx* ctx);
tt_status tt_ctx_get_stats(const tt_ctx* ctx, tt_stats* out);
void      tt_ctx_reset_stats(tt_ctx* ctx);
tt_precision tt_ctx_precision(const tt_ctx* ctx);

/* Limit, in SM clock cycles, of the bounded mbarrier waits of the
 * tensor-core row Gram (tt_gram_f32 with use_tensor_cores = 1, and the
 * Gram steps of TT-round that run on it); 0 restores the default of 4e9
 * cycles (about 2 s).  Every wait of that kernel gives up after the limit:
 * the kernel stops issuing work, lets the copies it already issued land and
 * waits for its MMAs (those two waits keep the default limit), frees its
 * tensor memory and returns; the call then fails with TT_ERR_TIMEOUT and
 * the context stays usable.  A limit far below the kernel's normal wait
 * times forces that path, for testing it.  Lanes created afterwards copy
 * the setting.  TT_ERR_ARG for a negative limit. */
tt_status tt_ctx_set_tc_wait_limit(tt_ctx* ctx, long long cycles);

/* Pipelined sweeps of TT-round (on != 0, the default; TTGB_PIPELINE=0 in
 * the environment turns them off for new contexts).  On a context that is
 * not a lane, with the series second pass on, a rounding runs each bond on
 * the assumption that its first Cholesky QR pass is healthy and its second
 * pass will be skipped: the factor is absorbed into the next core on a
 * high-priority stream as soon as the factorization ends, while the
 * product Q = L^{-1} X and the checks of the second pass run on a second
 * stream, and the host reads the checks once the next two bonds are
 * queued.  A bond that fails them is undone with the bonds queued after it
 * (the streams drain, the cores return to their buffers) and redone
 * sequentially, so the results are those of the sequential sweeps.  The
 * pipeline holds six more core-sized buffers; when
 * the context's HBM budget does not allow them the rounding runs
 * sequentially.  Profiling of every kernel family (tt_ctx_set_profiling
 * with no family set) runs sequentially too, so that each launch is timed
 * alone; timing one family keeps the pipeline, and its launches' events
 * are recorded on the stream each runs on.  The rounding stays ordered on the
 * context's stream: its internal streams wait for it and it waits for
 * them.  Lanes of tt_round_batched and of the server run the sequential
 * sweeps unless TTGB_LANE_PIPELINE=1 was set when the context was created
 * (the lanes already overlap whole roundings). */
tt_status tt_ctx_set_pipeline(tt_ctx* ctx, int on);

/* Enables (on != 0) or disables event timing of the library's launches. */
tt_status tt_ctx_set_profiling(tt_ctx* ctx, int on);
/* Restricts event timing to one kernel family (its name as reported by
 * tt_ctx_get_profile, copied); NULL or "" times every family again.  Two
 * events per timed launch cost host time, which shows in a step made of
 * many short launches; timing one family keeps that small. */
tt_status tt_ctx_set_profiling_family(tt_ctx* ctx, const char* family);
/* Synchronizes the stream and writes up to max_entries aggregated records
 * (one per kernel family, since the last reset) to out; *n_entries receives
 * the number of families. */
tt_status tt_ctx_get_profile(tt_ctx* ctx, tt_kernel_profile* out, int max_entries, int* n_entries);
void      tt_ctx_reset_profile(tt_ctx* ctx);

/* ---- tensors ---------------------------------------------------------- */

/* Creates a TT with d cores, mode sizes n[0..d-1] and ranks r[0..d]
 * (r[0] = r[d] = 1) in the context's storage type.  host_cores[k] points to
 * r[k]*n[k]*r[k+1] doubles in the [r][n][r] layout, copied to the device
 * (narrowed to FP32 on the device for FP32 contexts); host_cores == NULL
 * gives zeros.  The host arrays are read before the call returns. */
tt_status tt_tensor_create(tt_ctx* ctx, int d, const int* n, const int* r,
                           const double* const* host_cores, tt_tensor** out);

/* Wraps caller-owned device cores (dev_cores[k], [r][n][r] layout, dtype
 * `dtype`, which must be the context's storage type) without copying.  The
 * caller keeps ownership and must keep the memory alive until tt_tensor_free
 * of the wrapper. */
tt_status tt_tensor_wrap_device(tt_ctx* ctx, int d, const int* n, const int* r,
                                void* const* dev_cores, int dtype, tt_tensor** out);

/* d (if not NULL), n[0..d-1] and r[0..d] (if not NULL; caller-sized). */
tt_status tt_tensor_shape(const tt_tensor* x, int* d, int* n, int* r);

/* Device pointer of core k (for zero-copy readers). */
tt_status tt_tensor_core_ptr(const tt_tensor* x, int k, void** dev_ptr);

/* Copies the cores to host_cores[k] (r[k]*n[k]*r[k+1] doubles each;
 * FP32 storage is widened on the device first). */
tt_status tt_tensor_download(tt_ctx* ctx, const tt_tensor* x, double* const* host_cores);

/* As tt_tensor_create, but host_cores[k] already holds the core in the
 * context's storage type (float for TT_MIXED_TF32 and TT_FP32, double for
 * TT_FP64) and is copied without conversion.  From page-locked host memory
 * the copies are asynchronous on the context's stream: the host buffers must
 * stay unchanged until a later synchronizing call on the context returns
 * (tt_tensor_download*, tt_dot, tt_norm, tt_round ... all synchronize). */
tt_status tt_tensor_create_storage(tt_ctx* ctx, int d, const int* n, const int* r,
                                   const void* const* host_cores, tt_tensor** out);
/* Copies the cores to host_cores[k] in the storage type (no conversion) and
 * waits for the copies; page-locked buffers give full-bandwidth copies. */
tt_status tt_tensor_download_storage(tt_ctx* ctx, const tt_tensor* x, void* const* host_cores);

void tt_tensor_free(tt_tensor* x);

/* ---- TT arithmetic (Section 2) ---------------------------------------- */

/* out = sum_j alpha[j] x[j] by rank concatenation (Section 2: the k-th
 * TT-rank of x + y is r_k + s_k).  alpha is a host array of m doubles.
 * First core: [alpha_1 X_1 ... alpha_m X_m]; interior cores block diagonal;
 * last core stacked.  For d = 1 the single core is the linear combination. */
tt_status tt_add(tt_ctx* ctx, int m, const double* alpha,
                 const tt_tensor* const* x, tt_tensor** out);

/* out = alpha x (the last core scaled). */
tt_status tt_scale(tt_ctx* ctx, const tt_tensor* x, double alpha, tt_tensor** out);

/* <x, y> by the left-to-right contraction W_k = sum_i X_k(i)^T W_{k-1}
 * Y_k(i), W_0 = 1 (the inner product of Algorithms 1-8).  *out is a host
 * double. */
tt_status tt_dot(tt_ctx* ctx, const tt_tensor* x, const tt_tensor* y, double* out);

/* out[j] = <x, y[j]> for j < count, one contraction per pair, batched. */
tt_status tt_dot_many(tt_ctx* ctx, const tt_tensor* x, int count,
                      const tt_tensor* const* y, double* out);

/* ||x|| = ||core_1||_F after right-to-left orthogonalization of a copy
 * (no cancellation, unlike sqrt(<x, x>)). */
tt_status tt_norm(tt_ctx* ctx, const tt_tensor* x, double* out);

/* TT-round(x, delta) (Section 2): *out = x~ with ||x - x~|| <= delta ||x||.
 * Right-to-left orthogonalization of the right unfoldings by Cholesky QR
 * passes (Gram on the GPU, R factor absorbed into the left neighbour), then a
 * left-to-right sweep truncating each bond at eps = delta ||x|| / sqrt(d-1)
 * (minimal rank whose discarded singular values have root-sum-square
 * <= eps, never below 1).  d = 1 returns a copy.  err_est (may be NULL)
 * receives the root-sum-square of everything discarded, relative to ||x||.
 * The output's cores 1..d-1 are left-orthonormal. */
tt_status tt_round(tt_ctx* ctx, const tt_tensor* x, double delta,
                   tt_tensor** out, double* err_est);

/* tt_round that also copies the rounded cores to host memory in the storage
 * type: host_cores[k] must hold at least r[k]*n[k]*r[k+1] elements of x's
 * core k (rounding never raises a rank); on return it holds the rounded
 * core k, whose ranks *out reports.  Each core is copied as soon as the
 * left-to-right sweep has finished it, on a second stream, so from
 * page-locked memory the copies overlap the rest of the sweep; the call
 * returns when every copy is complete.  *out is the same device result as
 * tt_round's. */
tt_status tt_round_to_host(tt_ctx* ctx, const tt_tensor* x, double delta, tt_tensor** out,
                           double* err_est, void* const* host_cores);

/* Rounds count independent tensors, each at its own delta[i] (TT-round of
 * Section 2 applied to every x[i]; the paper has no batched form).  The
 * roundings run concurrently on the context's lanes (tt_ctx_set_concurrency):
 * child contexts with their own non-blocking streams, each driven by one
 * host thread (the calling thread drives lane 0), taking instances in
 * decreasing order of estimated work.  Lanes start after the work queued so
 * far on the context's stream and the stream continues after all of them,
 * so the call is stream-ordered like tt_round.  Each out[i] equals what
 * tt_round(ctx, x[i], delta[i]) returns (same kernels and decisions; lanes
 * share no workspace).  Device bytes of every lane count against the
 * context's HBM budget.  out[i] is set for every i, or all are NULL on
 * error (the first error seen is returned; the other lanes stop taking new
 * instances).  count = 0 is a no-op. */
tt_status tt_round_batched(tt_ctx* ctx, int count, const tt_tensor* const* x,
                           const double* delta, tt_tensor** out);

/* Number of lanes tt_round_batched uses (1 = sequential on the context's
 * stream; default 8; at most TT_MAX_LANES).  Lanes are created on first use
 * and live until the context is destroyed.  TT_ERR_ARG outside [1,
 * TT_MAX_LANES]. */
#define TT_MAX_LANES 64
tt_status tt_ctx_set_concurrency(tt_ctx* ctx, int lanes);
int       tt_ctx_get_concurrency(const tt_ctx* ctx);

/* TT-round(x, delta) with every TT-rank also capped at max_rank (the
 * rounding of the Krylov process of Section 4, where the accuracy is
 * replaced by a maximum TT-rank): each left-to-right bond keeps
 * min(max_rank, minimal rank within eps) singular values, so the error
 * bound delta ||x|| holds only when the cap does not bind; err_est reports
 * the discarded root-sum-square relative to ||x|| either way.  max_rank = 0
 * is tt_round; max_rank < 0 gives TT_ERR_ARG. */
tt_status tt_round_capped(tt_ctx* ctx, const tt_tensor* x, double delta, int max_rank,
                          tt_tensor** out, double* err_est);

/* TT-round(x, delta) from Gram matrices, without orthogonalizing the cores
 * (a GEMM-only variant of Section 2's TT-round): one right-to-left sweep of
 * contractions gives the Gram G_R of the right part of x at every bond;
 * then bond by bond, left to right, the Gram G_L of the current left
 * unfolding (the cores to its left are orthonormal by then), Cholesky
 * factors G_L = A A^T and G_R = B B^T (numerically zero pivots dropped),
 * the SVD A^T B = U S V^T (Jacobi, FP64 arithmetic), the truncation rank
 * from S at eps = delta ||x|| / sqrt(d - 1) (at most max_rank if > 0),
 * core_k <- core_k A^{-T} U_r and core_{k+1} <- S_r V_r^T B^{-1} core_{k+1}.
 * Squaring the condition numbers limits the accuracy to about
 * sqrt(r u) ||x|| (u the storage precision's unit round-off: FP64 contexts
 * resolve delta >= 1e-7 or so, FP32 ones delta >= 1e-3); err_est as
 * tt_round's.  Errors as tt_round; max_rank < 0 gives TT_ERR_ARG. */
tt_status tt_round_gram_svd(tt_ctx* ctx, const tt_tensor* x, double delta, int max_rank,
                            tt_tensor** out, double* err_est);

/* Randomized TT-rounding (randomize-then-orthogonalize; Section 2 cites it
 * for large tensors): omega is a TT with x's modes and ranks l_k whose
 * entries are the method's random draws (the caller draws them, e.g.
 * iid N(0,1)).  W_k = contraction of the right parts of x and omega at bond
 * k; then left to right the sketch Z = X_k^L W_{k+1} is orthonormalized
 * (a shifted Cholesky QR pass and two unshifted ones, so that Q spans
 * range(Z) whatever its conditioning), core_k <- Q and core_{k+1} <-
 * (Q^T X_k^L) core_{k+1}.  The ranks become min(l_k, rows of Z); with
 * probability near one the result is within a small factor of the best
 * approximation of those ranks once l_k exceeds the target rank by a few
 * (oversampling).  delta > 0: the result is then TT-rounded at delta.
 * TT_ERR_SHAPE when omega's modes differ from x's. */
tt_status tt_round_randomized(tt_ctx* ctx, const tt_tensor* x, const tt_tensor* omega, double delta,
                              tt_tensor** out);

/* ---- TT-matrices (Section 4) ------------------------------------------- */

/* A TT-matrix (TT-operator) M with M((i_1..i_d), (j_1..j_d)) =
 * M_1(i_1, j_1) ... M_d(i_d, j_d), core k stored [R_{k-1}][m_k][n_k][R_k]
 * row-major (R_k fastest; m_k output, n_k input mode size), R_0 = R_d = 1,
 * in the context's storage type.  Library-owned; released with
 * tt_operator_free.  The paper's experiments apply the Dirichlet Laplacian
 * in this form to build their inputs (Section 4). */
typedef struct tt_operator tt_operator;

/* Copies host FP64 cores (host_cores[k]: R[k]*m[k]*n[k]*R[k+1] doubles) to
 * the device (narrowed to FP32 for FP32 contexts), with the lists of each
 * core's nonzero entries per (a, i, b) triple that tt_matvec reads (built
 * on the host from the narrowed values).  TT_ERR_ARG for d < 1, R_0 != 1,
 * R_d != 1, or a size or rank < 1. */
tt_status tt_operator_create(tt_ctx* ctx, int d, const int* m, const int* n, const int* R,
                             const double* const* host_cores, tt_operator** out);
/* The d-dimensional Dirichlet Laplacian on n points per mode,
 * sum_k I x .. x L x .. x I with L = tridiag(-1, 2, -1) (grid scaling
 * dropped), as a TT-matrix of ranks 2: cores [L I], [[I 0], [L I]], [I; L]. */
tt_status tt_operator_laplacian(tt_ctx* ctx, int d, int n, tt_operator** out);
/* d, m[0..d-1], n[0..d-1], R[0..d] (each may be NULL; caller-sized). */
tt_status tt_operator_shape(const tt_operator* op, int* d, int* m, int* n, int* R);
/* Copies the cores to host FP64 arrays (layout as tt_operator_create). */
tt_status tt_operator_download(tt_ctx* ctx, const tt_operator* op, double* const* host_cores);
void      tt_operator_free(tt_operator* op);

/* y = M x: core k of y is y_k((a, p), i, (b, q)) = sum_j M_k(a, i, j, b)
 * x_k(p, j, q), mode sizes m_k and ranks R_k r_k (the operator's rank
 * index slowest).  Each output is the sum over the nonzero entries of its
 * triple (a, i, b) only, in the storage precision (FP32 contexts round at
 * FP32 level); zero entries cost nothing (a Laplacian core touches at most
 * three inputs per output).  TT_ERR_SHAPE when the orders or the input
 * modes differ; TT_ERR_ARG when a product rank R_k r_k exceeds 2^30 or an
 * operator core has more than 2^31 - 1 triples. */
tt_status tt_matvec(tt_ctx* ctx, const tt_operator* M, const tt_tensor* x, tt_tensor** out);

/* The input family of the paper's experiments (Section 4): from x_1,
 * a_j = y_j / ||y_j|| with y_j = tt_round_capped(x_j, delta, max_rank), and
 * x_{j+1} = -M a_j, for j = 1..m; out[0..m-1] receive a_1..a_m.  The paper
 * takes x_1 the all-ones tensor, M the Dirichlet Laplacian, delta = 0 and
 * max_rank = 1.  M must be square on x_1's modes (TT_ERR_SHAPE);
 * TT_ERR_BREAKDOWN if some y_j is zero. */
tt_status tt_krylov_basis(tt_ctx* ctx, const tt_operator* M, const tt_tensor* x1, int m, double delta,
                          int max_rank, tt_tensor** out);

/* ---- orthogonalization (Section 3) ------------------------------------ */

/* Orthogonalizes A[0..m-1] with `scheme` (Algorithms 1-5, 8) at rounding
 * accuracy delta.  Q[0..m-1] receive the basis (library-allocated), R
 * (host, m*m doubles, column-major) the upper triangular factor: column i
 * holds the coefficients of a_i, so a_i ~ sum_j R(j,i) q_j.  n_rounds (may
 * be NULL) receives the number of TT-round calls made.  TT_GRAM returns
 * TT_ERR_NOT_SPD when the Cholesky factorization of the Gram matrix fails
 * (remark on the Gram breakdown); a zero vector where a scheme normalises
 * gives TT_ERR_BREAKDOWN.  For TT_HOUSEHOLDER prod(n) must be >= m. */
tt_status tt_orthogonalize(tt_ctx* ctx, tt_scheme scheme, double delta,
                           tt_round_policy policy, int m,
                           const tt_tensor* const* A, tt_tensor** Q,
                           double* R, int* n_rounds);

/* The canonical basis TT-vector e_j (Section 3.3): rank 1, a single 1 at
 * the multi-index phi(j) with i_1 running fastest; j is 0-based
 * (0 <= j < prod n, else TT_ERR_ARG). */
tt_status tt_canonical(tt_ctx* ctx, int d, const int* n, long j, tt_tensor** out);

/* TT-Householder keeping only the Householder TT-vectors (Sections 4.4 and
 * 5: the basis q_k need not be formed): the first loop of Algorithm 8 with
 * its 3m roundings; U[0..m-1] receive u_1..u_m (library-allocated), R
 * (host, m*m, column-major) the upper triangular factor, n_rounds (may be
 * NULL) the roundings made.  Other arguments and errors as
 * tt_orthogonalize with TT_HOUSEHOLDER. */
tt_status tt_householder_vectors(tt_ctx* ctx, double delta, tt_round_policy policy, int m,
                                 const tt_tensor* const* A, tt_tensor** U, double* R, int* n_rounds);

/* Applies the reflections H_j = I - 2 u_j u_j^T of U[0..k-1] (Algorithm 7
 * each): transpose = 0 gives Q x = H_1 H_2 ... H_k x (H_k applied first),
 * transpose != 0 gives Q^T x = H_k ... H_1 x (H_1 first).  delta >= 0
 * TT-rounds after every reflection; delta < 0 rounds nothing (ranks add).
 * q_j of Algorithm 8 is tt_round(tt_householder_apply(U, j, e_j, 0, -1)).
 * k = 0 returns a copy of x. */
tt_status tt_householder_apply(tt_ctx* ctx, int k, const tt_tensor* const* U, const tt_tensor* x,
                               int transpose, double delta, tt_tensor** out);

/* ---- building block ---------------------------------------------------- */

/* Gram step of the Cholesky QR passes of TT-round: G = X X^T for a device
 * FP32 matrix X (n x K, row-major, leading dimension ldx >= K), written to
 * the device FP32 matrix G (n x n, row-major, overwritten).  Only tiles on
 * or below the diagonal are computed (128 x 128 tiles for the tensor-core
 * kernel, 64 x 64 for the CUDA-core one); strictly-upper tiles stay zero.
 * use_tensor_cores = 1 selects the tcgen05 kind::tf32 kernel (TMA-staged
 * operands, FP32 accumulation in TMEM), 0 the CUDA-core FP32 kernel.
 * use_tensor_cores = 2 computes the column Gram G = X^T X instead, X being
 * K x n row-major (ldx >= n): the Gram of a left unfolding, on tcgen05, the
 * operands transposed into K-major tiles on chip.
 * TT_ERR_ARG when the tensor-core kernel cannot take the layout (X not
 * 16-byte aligned or ldx*4 not a multiple of 16); TT_ERR_TIMEOUT when one of
 * its bounded waits ran out. */
tt_status tt_gram_f32(tt_ctx* ctx, int n, long K, const float* X, long ldx, float* G,
                      int use_tensor_cores);

/* Core-producing product of TT-round (apply Q = L^{-1} X, absorb
 * core <- core L): C = A op(B) for device FP32 matrices, A M x K row-major
 * (lda), op(B) = B^T with B N x K row-major when trans_b != 0, else B (K x N
 * row-major, ldb); C M x N row-major (ldc), overwritten.  use_tensor_cores
 * selects the kernel: 0 the CUDA-core FP32 kernel; 1 the tcgen05 kernel with
 * each operand split into three round-to-nearest TF32 parts (hi + mid + lo,
 * six products, FP32 accumulation: FP32-level accuracy); 2 the same with two
 * parts (hi + lo, three products, ~2^-22 relative error per product).  TT_ERR_ARG
 * when the tensor-core kernel cannot take the layout (a pointer or leading
 * dimension not 16-byte aligned). */
tt_status tt_gemm_f32(tt_ctx* ctx, int trans_b, int M, int N, int K, const float* A, long lda,
                      const float* B, long ldb, float* C, long ldc, int use_tensor_cores);

/* Factorization step of the Cholesky QR passes of TT-round:
 * G + s I = L L^T with s = shift_rel * trace(G), and T = L^{-1}.  A pivot
 * <= drop_rel * (max_j G_jj + s) marks its row of X as numerically dependent:
 * the column of L and the row and column of T are set to zero (*ndrop counts
 * them; host int, may be NULL).  G, L and T are device n x n row-major
 * matrices of the context's storage type (FP64, or FP32 for the other
 * precisions); only the lower triangle of G is read; L and T are lower
 * triangular on return.  Synchronizes the stream. */
tt_status tt_cholesky_inverse(tt_ctx* ctx, int n, const void* G, void* L, void* T,
                              double shift_rel, double drop_rel, int* ndrop);

/* Householder sign rule used by subsequent TT_HOUSEHOLDER calls. */
tt_status tt_set_sign_rule(tt_ctx* ctx, tt_sign_rule rule);

/* ---- allocation-free variant ------------------------------------------- */

/* <x, y> in FP64 without allocating any device memory, for callers that
 * cannot call cudaMalloc: hosts that hand all device memory to their own
 * pool up front (so a library allocation would fail or break their
 * accounting), and latency-critical loops that must not pay cudaMalloc's
 * implicit device synchronization.  The paper has no counterpart; this is the contraction of
 * tt_dot (W_k = sum_i X_k(i)^T W_{k-1} Y_k(i)) with its work arrays in a
 * static device array of 2^20 doubles (8 MiB) that every GPU loading the
 * library holds until the process exits.
 *
 * Arguments: cuda_stream (cudaStream_t, NULL = legacy default stream) on the
 * calling thread's current device; d, n[0..d-1], rx[0..d], ry[0..d] the
 * shapes (host arrays, boundary ranks 1); x_cores[k], y_cores[k] device
 * pointers (host arrays of them) to FP64 cores in the [r][n][r] layout;
 * result_dev a device pointer receiving the one double.  The call is
 * asynchronous on the stream: synchronize before reading result_dev.
 * Creates no context, allocates nothing, does not synchronize.
 *
 * The work arrays need max_k rx[k+1] ry[k+1] + max_k rx[k] n[k] ry[k+1]
 * doubles; larger shapes are rejected with TT_ERR_ARG (tt_last_error says
 * by how much).  The first call on a device looks up the array's device
 * address; make that first call before any stream capture.  All calls share
 * the one array, which keeps the previous call's contents: calls that
 * overlap on the GPU (different streams without ordering) race. */
tt_status tt_dot_f64_noalloc(void* cuda_stream, int d, const int* n, const int* rx, const int* ry,
                             const double* const* x_cores, const double* const* y_cores,
                             double* result_dev);

/* ---- request server ---------------------------------------------------- */

/* A request loop over one context (the paper has no counterpart: it is the
 * serving form of TT-round, Section 2, and of one outer iteration of the
 * Gram-Schmidt schemes, Algorithms 1-4, as an Arnoldi-type caller issues
 * them).  Requests of uneven order, mode size and rank are submitted at any
 * time from any host thread and run concurrently on `workers` lanes (child
 * contexts with their own non-blocking streams, one host thread each).
 * Admission is by device footprint: every request carries an upper bound
 * of the bytes it can hold at once (rounding workspace, output, the
 * concatenated sums of an orthogonalization step); a request starts only
 * while the admitted bounds sum to at most the footprint budget.  The
 * oldest waiting request keeps its place: a later one may start first only
 * if it fits beside the oldest one's bound.  Resident bases are copied to
 * the device once (tt_server_add_basis) and shared by all requests.
 *
 * Inputs belong to the server's context and must stay alive and unchanged
 * until their request is done; work queued on the context's stream before
 * tt_server_submit is complete before the request starts.  A result is
 * complete on the device when tt_server_wait returns it and belongs to the
 * caller (tt_tensor_free).  The context must not be destroyed before the
 * server.  Host faults are reported, never forced onto the GPU: a request
 * whose bound exceeds the budget is refused at submit (TT_ERR_OOM), a
 * queued one can be cancelled (TT_ERR_CANCELLED), a wait can time out
 * (TT_ERR_TIMEOUT, the ticket stays valid). */
typedef struct tt_server tt_server;

typedef enum { TT_REQ_ROUND = 0, TT_REQ_ORTH_STEP = 1 } tt_request_kind;

typedef struct {
    uint64_t submitted, completed, failed, cancelled, refused;
    uint64_t queued, running;          /* now */
    uint64_t footprint_in_use;         /* sum of the bounds of running requests */
    uint64_t footprint_peak;
    uint64_t footprint_budget;
    uint64_t roundings, kernel_launches, host_syncs;  /* work of completed requests */
} tt_server_stats;

/* workers in [1, TT_MAX_LANES]; footprint_budget in bytes (0: the
 * context's HBM budget, or no limit if it has none). */
tt_status tt_server_create(tt_ctx* ctx, int workers, size_t footprint_budget, tt_server** out);

/* Copies k >= 1 orthonormal TT tensors of equal modes into a resident
 * basis; *basis_id receives its handle.  The copies count against the
 * context's HBM budget.  Orthonormality is the caller's promise (Algorithms
 * 1-4 project on Q assuming Q^T Q = I). */
tt_status tt_server_add_basis(tt_server* s, int k, const tt_tensor* const* q, int* basis_id);

/* Queues a request and returns at once with *ticket.
 * TT_REQ_ROUND: TT-round(x, delta); basis_id, k and scheme are ignored.
 * TT_REQ_ORTH_STEP: one outer iteration of `scheme` (TT_CGS, TT_MGS, TT_CGS2
 * or TT_MGS2, rounding once per pass as in the paper's listings) for x
 * against the first k vectors of basis basis_id: the result is the new
 * normalised basis vector and the coefficients R(0..k, k+1).
 * TT_ERR_ARG / TT_ERR_SHAPE for bad arguments or modes that differ from the
 * basis; TT_ERR_OOM when the request's footprint bound exceeds the budget. */
tt_status tt_server_submit(tt_server* s, tt_request_kind kind, const tt_tensor* x, double delta, int basis_id,
                           int k, tt_scheme scheme, uint64_t* ticket);

/* Waits up to timeout_ms (< 0: no limit) for a request.  Returns the
 * request's own status (its message in tt_last_error), or TT_ERR_TIMEOUT
 * (ticket still valid), or TT_ERR_ARG for an unknown ticket.  Once a status
 * other than TT_ERR_TIMEOUT is returned the ticket is consumed.  out (may
 * be NULL: the result is then freed) receives the result; coef (may be
 * NULL) up to coef_cap doubles R(0..k, k+1) of an orthogonalization step;
 * times (may be NULL) 3 doubles: submit, start and finish instants in
 * seconds of the host's monotonic clock (CLOCK_MONOTONIC). */
tt_status tt_server_wait(tt_server* s, uint64_t ticket, int timeout_ms, tt_tensor** out, double* coef,
                         int coef_cap, double* times);

/* Removes a queued request (its wait then returns TT_ERR_CANCELLED).
 * TT_ERR_ARG if the ticket is unknown or the request has started. */
tt_status tt_server_cancel(tt_server* s, uint64_t ticket);

tt_status tt_server_get_stats(tt_server* s, tt_server_stats* out);

/* Cancels queued requests, waits for running ones, frees unclaimed results
 * and the bases, and stops the workers. */
void tt_server_destroy(tt_server* s);

/* ---- diagnostics ------------------------------------------------------- */

const char* tt_status_str(tt_status s);
/* Message of the last failed CUDA call on this thread ("" if none). */
const char* tt_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TTGB_H */
