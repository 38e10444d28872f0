// TT-matrices (TT-operators) and the TT matrix-vector product, with the
// Dirichlet Laplacian and the Krylov input family of the paper's experiments
// (Section 4: x_1 the all-ones tensor, a_j the normalised TT-round of x_j
// with the rank capped, x_{j+1} = -Delta_d a_j).
//
// A TT-matrix core k is stored [R_{k-1}][m_k][n_k][R_k] row-major (R_k
// fastest): M((i), (j)) = M_1(i_1, j_1) ... M_d(i_d, j_d).  The product
// y = M x has cores y_k((a, p), i, (b, q)) = sum_j M_k(a, i, j, b)
// x_k(p, j, q), ranks R_k r_k with the operator's rank index slowest.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "api_common.h"

struct tt_operator {
    tt_ctx* ctx = nullptr;
    int d = 0;
    std::vector<int> m, n, R;  // output modes, input modes, ranks (d + 1)
    tt_dtype dtype = TT_DTYPE_F64;
    std::vector<void*> cores;
    void* block = nullptr;
    size_t bytes = 0;
    size_t core_elems(int k) const { return (size_t)R[k] * m[k] * n[k] * R[k + 1]; }
};

namespace ttgb {

namespace {

// One CTA per (a, i, b) triple of the operator core and chunk of p: the
// nonzero entries M_k(a, i, j, b) over j are compacted into shared memory
// once (with their row offsets j Q into x), then every output
// y((a, p), i, (b, q)) of the chunk is their sum against x(p, j, q), in the
// storage precision.  Each thread produces V consecutive q at a time with
// one 16-byte load per entry and one 16-byte store (V = 4 for FP32, 2 for
// FP64 when Q and the core addresses allow it), running over q fastest, so
// the reads of x and the writes of y are coalesced; the operator is read
// once per CTA, and a zero entry costs nothing (the Laplacian's cores touch
// at most three inputs per output).  HBM-bound on the output, which is the
// product of the ranks.
template <class T, int V>
struct alignas(sizeof(T) * V) VecT {
    T v[V];
};

template <class T, int V>
__global__ void __launch_bounds__(256) matvec_core_kernel(const T* __restrict__ M, const T* __restrict__ X,
                                                          T* __restrict__ Y, int A, int P, int mo, int ni, int B,
                                                          int Q, int pchunk) {
    using VT = VecT<T, V>;
    extern __shared__ __align__(16) unsigned char mv_smem[];
    long long* offs = reinterpret_cast<long long*>(mv_smem);
    T* ms = reinterpret_cast<T*>(offs + ni);
    __shared__ int nnz_s;
    const long triples = (long)A * mo * B;
    const long BQ = (long)B * Q;
    const int Qv = Q / V;  // Q is a multiple of V
    const int p0 = blockIdx.y * pchunk, p1 = min(P, p0 + pchunk);
    // the thread's first (p, q) of the chunk and its stride, with q carried
    const int dq = (int)(blockDim.x % Qv), dp = (int)(blockDim.x / Qv);
    const int q0 = (int)(threadIdx.x % Qv), pp0 = p0 + (int)(threadIdx.x / Qv);
    for (long tr = blockIdx.x; tr < triples; tr += gridDim.x) {
        const int b = (int)(tr % B);
        const long ai = tr / B;
        const int i = (int)(ai % mo), a = (int)(ai / mo);
        __syncthreads();  // the previous triple's entries are no longer read
        if (threadIdx.x == 0) {
            int cnt = 0;
            const T* mrow = M + (((long)a * mo + i) * ni) * B + b;  // M[a, i, j, b] at mrow[j B]
            for (int j = 0; j < ni; ++j) {
                const T m = mrow[(long)j * B];
                if (m != T(0)) {
                    ms[cnt] = m;
                    offs[cnt] = (long long)j * Q;
                    ++cnt;
                }
            }
            nnz_s = cnt;
        }
        __syncthreads();
        const int nnz = nnz_s;
        T* yab = Y + (long)a * P * mo * BQ + (long)i * BQ + (long)b * Q;  // + p mo BQ + q
        int q = q0;
        for (int p = pp0; p < p1;) {
            const T* xp = X + (long)p * ni * Q + (long)q * V;
            VT acc;
#pragma unroll
            for (int l = 0; l < V; ++l) acc.v[l] = T(0);
            for (int t = 0; t < nnz; ++t) {
                const T m = ms[t];
                const VT xv = *reinterpret_cast<const VT*>(xp + offs[t]);
#pragma unroll
                for (int l = 0; l < V; ++l) acc.v[l] = fma(m, xv.v[l], acc.v[l]);
            }
            *reinterpret_cast<VT*>(yab + (long)p * mo * BQ + (long)q * V) = acc;
            q += dq;
            p += dp;
            if (q >= Qv) {
                q -= Qv;
                ++p;
            }
        }
    }
}

template <class T, int V>
void launch_matvec(Ctx& c, dim3 grid, size_t smem, const T* M, const T* X, T* Y, int A, int P, int mo, int ni,
                   int B, int Q, int pchunk) {
    matvec_core_kernel<T, V><<<grid, 256, smem, c.stream>>>(M, X, Y, A, P, mo, ni, B, Q, pchunk);
}

template <class T>
void matvec_core(Ctx& c, const T* M, const T* X, T* Y, int A, int P, int mo, int ni, int B, int Q) {
    const long total = (long)A * P * mo * B * Q;
    if (total == 0) return;
    const long triples = (long)A * mo * B;
    // about eight CTAs per SM in all: split p when the triples are fewer
    const long target = (long)std::max(1, c.sm_count) * 8;
    const int ysplit = (int)std::max(1L, std::min((long)P, (target + triples - 1) / triples));
    const int pchunk = (P + ysplit - 1) / ysplit;
    const dim3 grid((unsigned)std::min(triples, std::max(1L, target)), (unsigned)((P + pchunk - 1) / pchunk));
    const size_t smem = (size_t)ni * (sizeof(T) + sizeof(long long)) + 16;
    const double es = sizeof(T);
    ProfScope ps(c, sizeof(T) == 8 ? "matvec_f64" : "matvec_f32", 2.0 * (double)total * ni,
                 es * ((double)P * ni * Q + (double)A * mo * ni * B + (double)total));
    // 16-byte vectors when Q and both cores' addresses allow them
    const bool al16 = ((uintptr_t)X % 16 == 0) && ((uintptr_t)Y % 16 == 0);
    constexpr int V16 = 16 / sizeof(T);
    if (al16 && Q % V16 == 0)
        launch_matvec<T, V16>(c, grid, smem, M, X, Y, A, P, mo, ni, B, Q, pchunk);
    else if (sizeof(T) == 4 && al16 && Q % 2 == 0)
        launch_matvec<T, 2>(c, grid, smem, M, X, Y, A, P, mo, ni, B, Q, pchunk);
    else
        launch_matvec<T, 1>(c, grid, smem, M, X, Y, A, P, mo, ni, B, Q, pchunk);
    TT_LAUNCHED(c);
}

tt_operator* new_operator(tt_ctx* ctx, int d, const int* m, const int* n, const int* R) {
    if (d < 1 || !m || !n || !R) throw_status(TT_ERR_ARG, "d < 1 or NULL shape");
    if (R[0] != 1 || R[d] != 1) throw_status(TT_ERR_ARG, "R_0 and R_d must be 1");
    for (int k = 0; k < d; ++k)
        if (m[k] < 1 || n[k] < 1 || R[k + 1] < 1) throw_status(TT_ERR_ARG, "mode size or rank < 1");
    tt_operator* op = new tt_operator();
    op->ctx = ctx;
    op->d = d;
    op->m.assign(m, m + d);
    op->n.assign(n, n + d);
    op->R.assign(R, R + d + 1);
    op->dtype = storage_of(ctx->prec);
    const size_t es = dtype_size(op->dtype);
    std::vector<size_t> offs(d);
    size_t off = 0;
    for (int k = 0; k < d; ++k) {
        offs[k] = off;
        off += (op->core_elems(k) * es + 255) & ~size_t(255);
    }
    try {
        op->block = ctx->alloc(off);
    } catch (...) {
        delete op;
        throw;
    }
    op->bytes = off;
    op->cores.resize(d);
    for (int k = 0; k < d; ++k) op->cores[k] = (char*)op->block + offs[k];
    ctx->refs++;
    return op;
}

void free_operator(tt_operator* op) {
    if (!op) return;
    tt_ctx* c = op->ctx;
    c->release(op->block, op->bytes);
    delete op;
    drop_ctx_ref(c);
}

// uploads FP64 host cores, narrowed to the storage type on the host (the
// operators are small: a few ranks times n^2 per core)
void upload_cores(tt_operator* op, const double* const* host) {
    tt_ctx* c = op->ctx;
    for (int k = 0; k < op->d; ++k) {
        const size_t ne = op->core_elems(k);
        if (op->dtype == TT_DTYPE_F64) {
            TT_CUDA(cudaMemcpyAsync(op->cores[k], host[k], ne * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        } else {
            std::vector<float> f(host[k], host[k] + ne);
            TT_CUDA(cudaMemcpyAsync(op->cores[k], f.data(), ne * sizeof(float), cudaMemcpyHostToDevice, c->stream));
            c->sync();  // f is released at the end of this iteration
        }
    }
    c->sync();
}

tt_tensor* matvec_internal(tt_ctx* ctx, const tt_operator* op, const tt_tensor* x) {
    check_tensor(ctx, x);
    if (!op) throw_status(TT_ERR_ARG, "NULL operator");
    const Ctx* ho = op->ctx->root ? op->ctx->root : static_cast<const Ctx*>(op->ctx);
    const Ctx* hc = ctx->root ? ctx->root : static_cast<const Ctx*>(ctx);
    if (ho != hc) throw_status(TT_ERR_ARG, "operator belongs to another context");
    if (op->d != x->d) throw_status(TT_ERR_SHAPE, "orders differ");
    for (int k = 0; k < x->d; ++k) {
        if (op->n[k] != x->n[k]) throw_status(TT_ERR_SHAPE, "operator input modes differ from the tensor's");
        if (op->n[k] > 4096) throw_status(TT_ERR_ARG, "tt_matvec: input mode size above 4096");
        if ((long)x->r[k] * op->R[k] > 65535L * 1024) throw_status(TT_ERR_ARG, "tt_matvec: ranks too large");
    }
    const int d = x->d;
    std::vector<int> r(d + 1);
    for (int k = 0; k <= d; ++k) {
        const long rk = (long)op->R[k] * x->r[k];
        if (rk > (1L << 30)) throw_status(TT_ERR_ARG, "product rank too large");
        r[k] = (int)rk;
    }
    tt_tensor* y = new_tensor(ctx, d, op->m.data(), r.data());
    for (int k = 0; k < d; ++k) {
        if (ctx->prec == TT_FP64)
            matvec_core<double>(*ctx, (const double*)op->cores[k], (const double*)x->cores[k], (double*)y->cores[k],
                                op->R[k], x->r[k], op->m[k], op->n[k], op->R[k + 1], x->r[k + 1]);
        else
            matvec_core<float>(*ctx, (const float*)op->cores[k], (const float*)x->cores[k], (float*)y->cores[k],
                               op->R[k], x->r[k], op->m[k], op->n[k], op->R[k + 1], x->r[k + 1]);
    }
    return y;
}

// TT cores of Delta_d = sum_k I x .. x L x .. x I, L = tridiag(-1, 2, -1):
// first [L  I], interior [[I, 0], [L, I]], last [I; L] (ranks 2); d = 1: L.
std::vector<std::vector<double>> laplacian_cores(int d, int n, std::vector<int>& R) {
    auto Lij = [n](int i, int j) { return i == j ? 2.0 : (i - j == 1 || j - i == 1) ? -1.0 : 0.0; };
    auto Iij = [](int i, int j) { return i == j ? 1.0 : 0.0; };
    R.assign(d + 1, 2);
    R[0] = R[d] = 1;
    std::vector<std::vector<double>> cores(d);
    for (int k = 0; k < d; ++k) {
        const int A = R[k], B = R[k + 1];
        std::vector<double>& c = cores[k];
        c.assign((size_t)A * n * n * B, 0.0);
        auto at = [&](int a, int i, int j, int b) -> double& { return c[(((size_t)a * n + i) * n + j) * B + b]; };
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                if (d == 1) {
                    at(0, i, j, 0) = Lij(i, j);
                } else if (k == 0) {
                    at(0, i, j, 0) = Lij(i, j);
                    at(0, i, j, 1) = Iij(i, j);
                } else if (k == d - 1) {
                    at(0, i, j, 0) = Iij(i, j);
                    at(1, i, j, 0) = Lij(i, j);
                } else {
                    at(0, i, j, 0) = Iij(i, j);
                    at(1, i, j, 0) = Lij(i, j);
                    at(1, i, j, 1) = Iij(i, j);
                }
            }
    }
    return cores;
}

}  // namespace

}  // namespace ttgb

using namespace ttgb;

extern "C" {

tt_status tt_operator_create(tt_ctx* ctx, int d, const int* m, const int* n, const int* R,
                             const double* const* host_cores, tt_operator** out) {
    TT_API_BEGIN
    if (!ctx || !out || !host_cores) throw_status(TT_ERR_ARG, "NULL argument");
    *out = nullptr;
    for (int k = 0; k < d; ++k)
        if (!host_cores[k]) throw_status(TT_ERR_ARG, "NULL host core");
    tt_operator* op = new_operator(ctx, d, m, n, R);
    try {
        upload_cores(op, host_cores);
    } catch (...) {
        free_operator(op);
        throw;
    }
    *out = op;
    TT_API_END
}

tt_status tt_operator_laplacian(tt_ctx* ctx, int d, int n, tt_operator** out) {
    TT_API_BEGIN
    if (!ctx || !out || d < 1 || n < 1) throw_status(TT_ERR_ARG, "bad arguments");
    *out = nullptr;
    std::vector<int> R;
    std::vector<std::vector<double>> cores = laplacian_cores(d, n, R);
    std::vector<int> mm(d, n);
    tt_operator* op = new_operator(ctx, d, mm.data(), mm.data(), R.data());
    std::vector<const double*> ptrs(d);
    for (int k = 0; k < d; ++k) ptrs[k] = cores[k].data();
    try {
        upload_cores(op, ptrs.data());
    } catch (...) {
        free_operator(op);
        throw;
    }
    *out = op;
    TT_API_END
}

tt_status tt_operator_shape(const tt_operator* op, int* d, int* m, int* n, int* R) {
    if (!op) return TT_ERR_ARG;
    if (d) *d = op->d;
    for (int k = 0; k < op->d; ++k) {
        if (m) m[k] = op->m[k];
        if (n) n[k] = op->n[k];
    }
    if (R)
        for (int k = 0; k <= op->d; ++k) R[k] = op->R[k];
    return TT_OK;
}

tt_status tt_operator_download(tt_ctx* ctx, const tt_operator* op, double* const* host_cores) {
    TT_API_BEGIN
    if (!ctx || !op || !host_cores) throw_status(TT_ERR_ARG, "NULL argument");
    for (int k = 0; k < op->d; ++k) {
        const size_t ne = op->core_elems(k);
        if (op->dtype == TT_DTYPE_F64) {
            TT_CUDA(cudaMemcpyAsync(host_cores[k], op->cores[k], ne * sizeof(double), cudaMemcpyDeviceToHost,
                                    ctx->stream));
            ctx->sync();
        } else {
            std::vector<float> f(ne);
            TT_CUDA(cudaMemcpyAsync(f.data(), op->cores[k], ne * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
            ctx->sync();
            for (size_t e = 0; e < ne; ++e) host_cores[k][e] = f[e];
        }
    }
    TT_API_END
}

void tt_operator_free(tt_operator* op) { free_operator(op); }

tt_status tt_matvec(tt_ctx* ctx, const tt_operator* op, const tt_tensor* x, tt_tensor** out) {
    TT_API_BEGIN
    if (!ctx || !out) throw_status(TT_ERR_ARG, "NULL argument");
    *out = nullptr;
    *out = matvec_internal(ctx, op, x);
    TT_API_END
}

tt_status tt_krylov_basis(tt_ctx* ctx, const tt_operator* op, const tt_tensor* x1, int m, double delta,
                          int max_rank, tt_tensor** out) {
    TT_API_BEGIN
    if (!ctx || !out || m < 1 || max_rank < 0) throw_status(TT_ERR_ARG, "bad arguments");
    for (int j = 0; j < m; ++j) out[j] = nullptr;
    check_tensor(ctx, x1);
    if (!op) throw_status(TT_ERR_ARG, "NULL operator");
    for (int k = 0; k < x1->d; ++k)
        if (op->d != x1->d || op->m[k] != op->n[k] || op->n[k] != x1->n[k])
            throw_status(TT_ERR_SHAPE, "the Krylov process needs a square operator on the tensor's modes");
    std::vector<TensorGuard> A(m);
    TensorGuard xg;  // x_{j+1} (x_1 is borrowed)
    const tt_tensor* x = x1;
    for (int j = 0; j < m; ++j) {
        TensorGuard y(round_internal(ctx, x, delta, nullptr, nullptr, max_rank));
        const double nrm = norm_internal(ctx, y.get());
        if (!(nrm > 0.0) || !isfinite(nrm)) throw_status(TT_ERR_BREAKDOWN, "zero Krylov vector");
        A[j].reset(scale_internal(ctx, y.get(), 1.0 / nrm));
        if (j + 1 < m) {
            TensorGuard ax(matvec_internal(ctx, op, A[j].get()));
            xg.reset(scale_internal(ctx, ax.get(), -1.0));
            x = xg.get();
        }
    }
    for (int j = 0; j < m; ++j) out[j] = A[j].release();
    TT_API_END
}

}  // extern "C"
