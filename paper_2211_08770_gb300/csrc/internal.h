// Internal interfaces of the TT library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ttgb.h"

namespace ttgb {

// ---------------------------------------------------------------- errors
struct Error {
    tt_status status;
    std::string msg;
};
[[noreturn]] void throw_status(tt_status s, const std::string& msg);
[[noreturn]] void throw_cuda(cudaError_t e, const char* what, const char* file, int line);
#define TT_CUDA(x)                                                          \
    do {                                                                    \
        cudaError_t e__ = (x);                                              \
        if (e__ != cudaSuccess) ::ttgb::throw_cuda(e__, #x, __FILE__, __LINE__); \
    } while (0)
// after every kernel launch: catches launch-configuration errors at once
#define TT_LAUNCHED(ctx)                                                    \
    do {                                                                    \
        (ctx).stats.kernel_launches++;                                      \
        cudaError_t e__ = cudaGetLastError();                               \
        if (e__ != cudaSuccess) ::ttgb::throw_cuda(e__, "kernel launch", __FILE__, __LINE__); \
    } while (0)

// Raises a kernel's dynamic shared-memory limit once per process; safe when
// several host threads (batched rounding, serving workers) launch at once.
// It is set for the device current at the first call (one device per
// process: multi-GPU runs are independent replicas).
template <class F>
void set_smem_once(std::atomic<bool>& flag, F* func, int bytes) {
    if (flag.load(std::memory_order_acquire)) return;
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    if (flag.load(std::memory_order_relaxed)) return;
    cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) throw_cuda(e, "cudaFuncSetAttribute", __FILE__, __LINE__);
    flag.store(true, std::memory_order_release);
}

// ---------------------------------------------------------------- kernels
// Small-matrix factorization status written by the Cholesky kernel.
struct CholStatus {
    int ndrop;          // pivots dropped as numerically dependent
    int nonfinite;      // NaN/Inf met
    double min_ratio;   // min over kept j of pivot_j / (G_jj + shift)
    double trace;       // trace(G) (before shift)
    double max_diag;    // max_j G_jj (before shift)
};

struct Ctx;

// Known zero structure of op(A) (M x K) and op(B) (K x N) in a product:
// each output tile then contracts only over the k-range where both can be
// non-zero.  Only products with exact zeros are left out, so the result is
// the same for finite data (the triangular factors and inverses of the
// Cholesky QR passes).
enum : int {
    TRI_A_LOWER = 1,  // op(A)(m, k) = 0 for k > m
    TRI_A_UPPER = 2,  // op(A)(m, k) = 0 for k < m
    TRI_B_LOWER = 4,  // op(B)(k, n) = 0 for k < n
    TRI_B_UPPER = 8,  // op(B)(k, n) = 0 for k > n
    TRI_C_LOWER = 16, // only the lower triangle of C is computed and written:
                      // output tiles strictly above the diagonal are skipped
                      // and elements above it are left unchanged
};

// the k-range [kb, ke) an output tile (rows m0.., cols n0..) needs; an
// unwanted tile (TRI_C_LOWER) gets an empty range and writes nothing
__host__ __device__ inline bool tri_skip_tile(int tri, long m0, long n0, long bm) {
    return (tri & TRI_C_LOWER) && n0 >= m0 + bm;
}
__host__ __device__ inline void tri_krange(int tri, long m0, long n0, long bm, long bn, long& kb, long& ke) {
    if (tri & TRI_A_LOWER) ke = ke < m0 + bm ? ke : m0 + bm;
    if (tri & TRI_A_UPPER) kb = kb > m0 ? kb : m0;
    if (tri & TRI_B_LOWER) kb = kb > n0 ? kb : n0;
    if (tri & TRI_B_UPPER) ke = ke < n0 + bn ? ke : n0 + bn;
}

// Algorithmic flops of one product with the TRI_* zero structure: twice
// the multiply-adds with both factors possibly non-zero (2MNK when dense).
double gemm_flops(long M, long N, long K, int tri);

// C = alpha op(A) op(B) + beta C, row-major with leading dimensions.
// op(A) is M x K, op(B) is K x N.  batch > 1: blockIdx.z strides.  tri:
// TRI_* flags of the operands' zero structure.
template <class T>
void gemm(Ctx& c, bool tA, bool tB, int M, int N, int K, T alpha, const T* A, long lda,
          const T* B, long ldb, T beta, T* C, long ldc, int batch = 1, long sA = 0,
          long sB = 0, long sC = 0, int tri = 0);

// G (n x n, row-major, lower triangle written, type S) = X X^T when rows,
// i.e. X is n x K row-major (ldx) and the contraction runs over K; or
// X^T X when !rows, X is K x n row-major and the contraction runs over rows.
// G is overwritten.  Split-K with atomics; FP accumulation in T.
template <class T, class S>
void gram(Ctx& c, bool rows, int n, long K, const T* X, long ldx, S* G);

// Cholesky factorization with rank drop and the explicit inverse of the
// factor: G + shift I = L L^T, T = L^{-1}, all n x n row-major (lower
// triangles; upper parts written as zeros), compute type C.
// shift = shift_rel * trace(G).  Pivots <= drop_rel * (max_j G_jj + shift)
// are dropped: the column of L and the row and column of T are zero.
// One CTA with everything in shared memory for n <= chol_tile_max(), else
// blockwise with block size Ctx::chol_nb, or a fixed per-order table.
template <class S, class C>
void chol_inv(Ctx& c, int n, const S* G, S* L, S* T, double shift_rel, double drop_rel, CholStatus* st_dev);
// the same with a given block size (nb >= n: the one-CTA kernel)
template <class S, class C>
void chol_inv_nb(Ctx& c, int n, int nb, const S* G, S* L, S* T, double shift_rel, double drop_rel,
                 CholStatus* st_dev);
template <class S, class C>
int chol_tile_max();

// One-sided Jacobi SVD of the rows of R (p x b, row-major, p <= b):
// R = U diag(sigma) V^T.  Outputs U (p x p, row-major, columns sorted by
// decreasing sigma), SVt (p x b, row-major, row i = sigma_i v_i^T, sorted),
// sigma (p doubles, sorted).  work: p*b + p*p doubles (W, U^T), FP64
// arithmetic.  A pair of rows is left alone when |<x,y>| <= tol ||x|| ||y||
// or when one row's norm is <= floor_rel ||R||_F (noise of the larger rows).
// Rotations are exact orthogonal transforms, so U diag(sigma) V^T = R up to
// rounding whatever the tolerance: the discarded rows' norms are exactly the
// truncation error, and the tolerance only affects how close to optimal the
// ranks are.
template <class S>
void jacobi_svd(Ctx& c, int p, int b, const S* R, S* U, S* SVt, double* sigma, S* work, double tol,
                double floor_rel);

// FP32 one-sided Jacobi on the columns of R for FP32 data: W (nr x len,
// row-major, ld_src) holds the columns of R as rows; on return sigma (nr
// doubles, device) holds the column norms of the orthogonalized R sorted
// decreasingly and U (len x nr, row-major) the matching unit columns
// (orthogonal to about tol; callers re-orthonormalize what they keep).
// Wwork: nr x round_up(len, 4) floats.  False (nothing launched) when the
// rows do not fit one thread-block cluster's shared memory.
bool jacobi_cols_f32(Ctx& c, int nr, int len, const float* Wsrc, long ld_src, float* Wwork, float* U,
                     double* sigma, double tol, double floor_rel);

// sum of squares of n elements, FP64 accumulation, written to *out (device).
template <class T>
void sumsq(Ctx& c, long n, const T* x, double* out);

// Frobenius norms for the sigma_min certificate of a lower-triangular L
// with inverse T: out[0] += ||T||_F^2, out[1] += ||L - I||_F^2.
template <class S>
void inv_and_identity_defect(Ctx& c, int n, const S* L, const S* T, double* out);

// Near-identity symmetric G (n x n, lower triangle valid): E = G - I
// (symmetric, full) and ||E||_F^2 into *dev_out (FP64 accumulation).
template <class T>
void near_identity(Ctx& c, int n, const T* G, T* E, double* dev_out);
// Truncated Taylor series of order m (1..3) in the symmetric E:
// S = (I + E)^(-1/2) over E and R = (I + E)^(1/2) into R; E2 = E^2 is read
// when m >= 2 and E3 = E^3 when m >= 3 (R may alias E2).  When e2max is
// given, *e2max becomes max(*e2max, *e2) (device scalars: ||E||_F^2 of this
// pass and the running maximum).
template <class T>
void poly_pair(Ctx& c, int n, int m, T* E, const T* E2, const T* E3, T* R, const double* e2 = nullptr,
               double* e2max = nullptr);

template <class T>
void fill_identity(Ctx& c, int n, T* A, long lda);  // A (n x n) = I
template <class T>
void scale_inplace(Ctx& c, long n, T* x, double alpha);
template <class Tin, class Tout>
void convert(Ctx& c, long n, const Tin* x, Tout* y);
// Y (rows x cols) = X^T where X is cols x rows, both row-major
template <class T>
void transpose(Ctx& c, int rows, int cols, const T* X, T* Y);

// block copy for the rank-concatenating sum: up to 64 blocks per launch,
// passed by value as a kernel parameter (no host-to-device copy).
struct BlockDesc {
    const void* src;  // a x n x b source core
    long dst_off;     // element offset of block (oa, 0, ob) in the destination
    int a, b;
    double alpha;
};
struct BlockList {
    BlockDesc blk[64];
    int count;
};
template <class T>
void scatter_blocks(Ctx& c, const BlockList& list, int n, long dst_ld_b, long dst_ld_row, T* dst,
                    int max_a, int max_b);
template <class T>
void axpy(Ctx& c, long n, double alpha, const T* x, T* y);  // y += alpha x

// FP32 CUDA-core GEMM / split-K Gram with 128 x 128 tiles (same contracts
// as gemm() and gram()); false (nothing launched) when a pointer is not
// 16-byte aligned or a leading dimension (batch stride) not a multiple of 4.
bool sgemm(Ctx& c, bool tA, bool tB, int M, int N, int K, float alpha, const float* A, long lda, const float* B,
           long ldb, float beta, float* C, long ldc, int batch, long sA, long sB, long sC, int tri = 0);
bool sgram(Ctx& c, bool rows, int n, long K, const float* X, long ldx, float* G);

// tcgen05 TF32 Gram of the rows of X (n x K, row-major): G = X X^T (lower
// tiles), split-K, FP32 accumulation in TMEM, atomically added into G (FP32,
// zeroed first).  Returns false when the shape is not supported.
bool gram_rows_tc_tf32(Ctx& c, int n, long K, const float* X, long ldx, float* G);
// G = X^T X for X (m x n, row-major, ldx): the column Gram, same kernel family
// (operands transposed into K-major tiles by converter warps).
bool gram_cols_tc_tf32(Ctx& c, int n, long m, const float* X, long ldx, float* G);
// C (M x N, row-major, ldc) = A (M x K, row-major) op(B), op(B) = B^T with B
// N x K row-major when bT, else B (K x N row-major); split-TF32 on tcgen05
// with FP32 accumulation: nsplit = 3 (hi + mid + lo, 6 MMAs per k-step,
// FP32-level products) or 2 (hi + lo, 3 MMAs).  Returns false (nothing
// launched) when a pointer or leading dimension is not 16-byte aligned.
bool gemm_tc3_tf32(Ctx& c, bool bT, int M, int N, int K, const float* A, long lda, const float* B, long ldb,
                   float* C, long ldc, int nsplit);
// Triangular solve with a lower-triangular a x a L (leading dimension a):
// rows: Q (a x K) = L^{-1} X; !rows: Q (K x a) = X L^{-T}; row-major, Q does
// not alias X.  Blocked forward substitution (backward stable), FP64
// arithmetic in the diagonal blocks; a zero pivot gives a zero component.
template <class T>
void trsm_lower(Ctx& c, bool rows, int a, long K, const T* L, const T* X, T* Q);

// reads (and clears) the tensor-core timeout flag; throws TT_ERR_TIMEOUT if set
void check_tc_error(Ctx& c);

// ---------------------------------------------------------------- context
struct ProfRec {
    int fam;
    double flops, bytes;
    cudaEvent_t a, b;
};

struct Ctx {
    int device = 0;
    tt_precision prec = TT_FP64;
    cudaStream_t stream = nullptr;
    size_t budget = 0;
    tt_stats stats{};
    tt_sign_rule sign_rule = TT_SIGN_STABLE;
    int sm_count = 0;
    bool use_tc = true;       // tensor-core Gram in TT_MIXED_TF32
    // tensor-core split-TF32 apply / absorb GEMMs in TT_MIXED_TF32 (opt-in:
    // the tensor cores' FP32 accumulation truncates, and the apply Q = L^{-1} X
    // cancels heavily, so a full rounding lands near 2.5e-6 relative error at
    // delta = 1e-6 against 1.06e-6 with the CUDA-core FP32 GEMM)
    bool use_tc_gemm = false;
    int tc_gemm_split = 3;    // 3: hi + mid + lo (6 products), 2: hi + lo (3 products)
    // the absorbs alone (core_{k-1} L, R core_{k+1}: no explicit inverse, no
    // cancellation) on the split-TF32 tensor-core GEMM
    bool use_tc_absorb = false;
    int* tc_err = nullptr;  // device flag: a bounded wait of a tensor-core kernel ran out
    long long tc_wait_limit = 0;  // SM cycles of the row Gram's bounded waits (0: ~2 s)
    // lifetime: one reference for the owner plus one per live tensor; the
    // context is deleted when the last reference goes
    std::atomic<long> refs{1};

    // Lanes: child contexts with their own non-blocking streams that run
    // independent roundings concurrently (batched rounding, serving).  A
    // lane's device bytes are charged to its root's budget and counters.
    Ctx* root = nullptr;          // non-null for a lane
    bool owns_stream = false;     // lanes create (and destroy) their stream
    std::mutex acct_mu;           // guards stats.bytes_in_use / peak_bytes of a root
    std::vector<Ctx*> lanes;      // lanes owned by this root (created on demand)
    int max_lanes = 8;            // concurrency of tt_round_batched
    int chol_nb = 0;              // block size of chol_inv (0: the per-order table)
    int colgram_stages = 5;       // raw staging stages of the tensor-core column Gram (3 or 5)
    bool use_series = true;       // series second pass of Cholesky QR when it is accurate
    bool series_force_retry = false;  // treat series passes as invalid (tests the retry)
    bool series_no_skip = false;      // run every second pass (tests the series pass itself)

    cudaStream_t copy_stream = nullptr;  // device-to-host copies overlapping the
                                         // left-to-right sweep (created on first use)
    // Pipelined sweeps of TT-round (root contexts; off while profiling):
    // the critical path (Gram, Cholesky, absorb) runs on a high-priority
    // stream, the applies and second-pass checks on a second stream, and
    // the host reads each bond's decision from page-locked words
    bool pipeline = true;
    bool lane_pipeline = false;  // lanes (batched, serving) pipeline their roundings too
    // when set, the next chol_inv records it on the stream just before its
    // first single-CTA tile kernel (after the factor's preparation), then
    // clears it: the pipelined sweeps release the previous bond's checks
    // there, so the tile kernel holds its SM before they fill the GPU
    cudaEvent_t chol_mark = nullptr;
    // when set, a blocked chol_inv computes the off-diagonal blocks of the
    // inverse on this stream (after L is final) instead of the context's
    cudaStream_t chol_tail = nullptr;
    // when set, a blocked chol_inv records it just before its last tile
    // kernel, when L's columns left of the last block (the first chol_split
    // columns) are final, sets chol_split and clears it; the pipelined
    // sweeps start the absorb's product with those columns there, beside
    // the last tile kernel
    cudaEvent_t chol_mark2 = nullptr;
    int chol_split = 0;
    cudaStream_t crit_stream = nullptr;
    cudaStream_t side_stream = nullptr;
    cudaStream_t tail_stream = nullptr;  // the factorizations' inverse tails
    cudaStream_t crit2_stream = nullptr; // high priority, beside the critical stream
    void* host_words = nullptr;  // kHostWords bytes, page-locked
    static constexpr size_t kHostWords = 4096;

    // event profiling of launches (off by default)
    bool prof = false;
    int prof_nest = 0;            // open ProfScopes: only the outermost records
    std::string prof_only;        // time only this family ("" = all)
    std::vector<std::string> fam_names;
    std::vector<ProfRec> recs;
    std::vector<cudaEvent_t> ev_pool;

    cudaStream_t copies();  // copy_stream, created on first use
    cudaStream_t crit();    // crit_stream, created on first use
    cudaStream_t side();    // side_stream, created on first use
    cudaStream_t tail();    // tail_stream, created on first use
    cudaStream_t crit2();   // crit2_stream, created on first use
    void* pinned_words();   // host_words, allocated on first use
    void* alloc(size_t bytes);
    void release(void* p, size_t bytes);
    void sync();
    int family(const char* name);
    cudaEvent_t event();
    ~Ctx();
};

// Returns the root's lanes [0, count), creating missing ones (stream,
// status word, settings copied from the root).
std::vector<Ctx*> get_lanes(Ctx& root, int count);
// Adds a lane's counters (all but the byte counters, kept by the root) and
// event-profile records into the root, then clears them on the lane.
void merge_lane(Ctx& root, Ctx& lane);

// Records CUDA events on the context stream around the launches made while
// it is alive, when profiling is on.
struct ProfScope {
    Ctx& c;
    int fam = -1;
    double flops, bytes;
    cudaEvent_t a = nullptr;
    ProfScope(Ctx& ctx, const char* name, double fl, double by);
    ~ProfScope();
};

}  // namespace ttgb
