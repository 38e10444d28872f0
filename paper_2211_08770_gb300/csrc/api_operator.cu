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
    // the nonzero entries of each core, listed per (a, i, b) triple (built
    // on the host at upload): entries ptr[t] .. ptr[t + 1] - 1 of triple
    // t = (a m_k + i) R_k + b have input index js[e] and value vals[e]
    std::vector<const int*> nz_ptr, nz_j;
    std::vector<const void*> nz_val;
    std::vector<long> nz_count;  // entries per core
    void* nz_block = nullptr;
    size_t nz_bytes = 0;
    size_t core_elems(int k) const { return (size_t)R[k] * m[k] * n[k] * R[k + 1]; }
};

namespace ttgb {

namespace {

// y((a, p), i, (b, q)) = sum_j M_k(a, i, j, b) x(p, j, q) over the nonzero
// M_k(a, i, j, b) only (the lists built at upload; the Laplacian's cores
// have at most three per triple), in the storage precision.  A work item is
// one triple and a chunk of rows p; a grid of resident CTAs takes the items
// in turn, all triples of a chunk before the next chunk.  Each thread produces V consecutive q at a time with one 16-byte
// load per entry and one 16-byte store (V = 4 for FP32, 2 for FP64 when Q
// and the core addresses allow it), two such vectors per iteration, running
// over q fastest, so the reads of x and the writes of y are coalesced and
// every thread has two independent loads in flight; the entry lists are
// uniform across the CTA (broadcast loads).  HBM-bound on the output, which
// is the product of the ranks.
template <class T, int V>
struct alignas(sizeof(T) * V) VecT {
    T v[V];
};

constexpr int kMvThreads = 256;

template <class T, int V>
__global__ void __launch_bounds__(kMvThreads) matvec_core_kernel(const int* __restrict__ nzp,
                                                                 const int* __restrict__ nzj,
                                                                 const T* __restrict__ nzv, const T* __restrict__ X,
                                                                 T* __restrict__ Y, int P, int mo, int ni, int B,
                                                                 int Q, int pchunk, int triples, int items) {
    using VT = VecT<T, V>;
    const long BQ = (long)B * Q;
    const int Qv = Q / V;  // Q is a multiple of V
    // the thread's first (p, q) of a chunk and its stride, with q carried
    const int dq = kMvThreads % Qv, dp = kMvThreads / Qv;
    const int q0 = (int)threadIdx.x % Qv, pr0 = (int)threadIdx.x / Qv;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        // chunk-major: the CTAs resident at a time share a few chunks of
        // rows of x, which stay in L2 while every triple reads them
        const int ch = it / triples;
        const int tr = it - ch * triples;
        const int b = tr % B;
        const int ai = tr / B;
        const int i = ai % mo, a = ai / mo;
        const int e0 = nzp[tr], nnz = nzp[tr + 1] - e0;
        const int p1 = min(P, (ch + 1) * pchunk);
        const long P_mo_BQ = (long)P * mo * BQ;
        T* yab = Y + a * P_mo_BQ + (long)i * BQ + (long)b * Q;  // + p mo BQ + q
        int q = q0, p = ch * pchunk + pr0;
        while (p < p1) {
            int q2 = q + dq, p2 = p + dp;
            if (q2 >= Qv) {
                q2 -= Qv;
                ++p2;
            }
            const bool two = p2 < p1;
            const T* x1 = X + (long)p * ni * Q + (long)q * V;
            const T* x2 = X + (long)p2 * ni * Q + (long)q2 * V;
            VT acc1, acc2;
#pragma unroll
            for (int l = 0; l < V; ++l) acc1.v[l] = acc2.v[l] = T(0);
            for (int t = 0; t < nnz; ++t) {
                const T m = nzv[e0 + t];
                const long off = (long)nzj[e0 + t] * Q;
                const VT u = *reinterpret_cast<const VT*>(x1 + off);
                VT w;
                if (two) w = *reinterpret_cast<const VT*>(x2 + off);
#pragma unroll
                for (int l = 0; l < V; ++l) acc1.v[l] = fma(m, u.v[l], acc1.v[l]);
                if (two) {
#pragma unroll
                    for (int l = 0; l < V; ++l) acc2.v[l] = fma(m, w.v[l], acc2.v[l]);
                }
            }
            *reinterpret_cast<VT*>(yab + (long)p * mo * BQ + (long)q * V) = acc1;
            if (two) *reinterpret_cast<VT*>(yab + (long)p2 * mo * BQ + (long)q2 * V) = acc2;
            q = q2 + dq;
            p = p2 + dp;
            if (q >= Qv) {
                q -= Qv;
                ++p;
            }
        }
    }
}

template <class T, int V>
void launch_matvec(Ctx& c, const int* nzp, const int* nzj, const T* nzv, const T* X, T* Y, int P, int mo, int ni,
                   int B, int Q, long triples) {
    // resident CTAs of this kernel on the whole GPU
    static const int per_sm = [] {
        int nb = 0;
        TT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, matvec_core_kernel<T, V>, kMvThreads, 0));
        return std::max(1, nb);
    }();
    const long slots = (long)std::max(1, c.sm_count) * per_sm;
    // items of about four 256-vector steps each, at least eight per
    // resident CTA where the rows allow it (the last round of items is then
    // a small part of the launch)
    const long vecs = (long)P * (Q / V);
    int nch = (int)std::max(1L, std::min((long)P, (vecs + 4L * kMvThreads - 1) / (4L * kMvThreads)));
    if (triples * nch < 8 * slots) nch = (int)std::min((long)P, (8 * slots + triples - 1) / triples);
    nch = (int)std::max(1L, std::min((long)nch, (long)INT32_MAX / triples));
    const int pchunk = (P + nch - 1) / nch;
    nch = (P + pchunk - 1) / pchunk;
    const long items = triples * nch;  // <= INT_MAX (checked by the caller)
    const unsigned grid = (unsigned)std::min(items, slots);
    matvec_core_kernel<T, V><<<grid, kMvThreads, 0, c.stream>>>(nzp, nzj, nzv, X, Y, P, mo, ni, B, Q, pchunk,
                                                               (int)triples, (int)items);
}

template <class T>
void matvec_core(Ctx& c, const int* nzp, const int* nzj, const T* nzv, long nnz, const T* X, T* Y, int A, int P,
                 int mo, int ni, int B, int Q) {
    const long total = (long)A * P * mo * B * Q;
    if (total == 0) return;
    const long triples = (long)A * mo * B;
    const double es = sizeof(T);
    ProfScope ps(c, sizeof(T) == 8 ? "matvec_f64" : "matvec_f32", 2.0 * (double)nnz * P * Q,
                 es * ((double)P * ni * Q + (double)total) + (es + 4.0) * nnz + 4.0 * (triples + 1));
    // 16-byte vectors when Q and both cores' addresses allow them
    const bool al16 = ((uintptr_t)X % 16 == 0) && ((uintptr_t)Y % 16 == 0);
    constexpr int V16 = 16 / sizeof(T);
    if (al16 && Q % V16 == 0)
        launch_matvec<T, V16>(c, nzp, nzj, nzv, X, Y, P, mo, ni, B, Q, triples);
    else if (sizeof(T) == 4 && al16 && Q % 2 == 0)
        launch_matvec<T, 2>(c, nzp, nzj, nzv, X, Y, P, mo, ni, B, Q, triples);
    else
        launch_matvec<T, 1>(c, nzp, nzj, nzv, X, Y, P, mo, ni, B, Q, triples);
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
    if (op->nz_block) c->release(op->nz_block, op->nz_bytes);
    delete op;
    drop_ctx_ref(c);
}

// uploads FP64 host cores, narrowed to the storage type on the host (the
// operators are small: a few ranks times n^2 per core), and the lists of
// each core's nonzero entries (of the narrowed values) per (a, i, b) triple
template <class T>
void upload_t(tt_operator* op, const double* const* host) {
    tt_ctx* c = op->ctx;
    const int d = op->d;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    std::vector<std::vector<T>> vals(d), narrowed(d);
    std::vector<std::vector<int>> ptr(d), js(d);
    size_t nzb = 0;
    for (int k = 0; k < d; ++k) {
        const int A = op->R[k], mo = op->m[k], ni = op->n[k], B = op->R[k + 1];
        const size_t ne = op->core_elems(k);
        narrowed[k].assign(host[k], host[k] + ne);
        const std::vector<T>& h = narrowed[k];
        const long triples = (long)A * mo * B;
        ptr[k].assign(triples + 1, 0);
        for (int a = 0; a < A; ++a)
            for (int i = 0; i < mo; ++i)
                for (int b = 0; b < B; ++b) {
                    const long t = ((long)a * mo + i) * B + b;
                    for (int j = 0; j < ni; ++j) {
                        const T v = h[(((size_t)a * mo + i) * ni + j) * B + b];
                        if (v != T(0)) {
                            vals[k].push_back(v);
                            js[k].push_back(j);
                        }
                    }
                    if (vals[k].size() > (size_t)INT32_MAX) throw_status(TT_ERR_ARG, "operator core too large");
                    ptr[k][t + 1] = (int)vals[k].size();
                }
        nzb += al(ptr[k].size() * sizeof(int)) + al(std::max<size_t>(1, js[k].size()) * sizeof(int)) +
               al(std::max<size_t>(1, vals[k].size()) * sizeof(T));
    }
    op->nz_block = c->alloc(nzb);
    op->nz_bytes = nzb;
    op->nz_ptr.resize(d);
    op->nz_j.resize(d);
    op->nz_val.resize(d);
    op->nz_count.resize(d);
    char* p = (char*)op->nz_block;
    for (int k = 0; k < d; ++k) {
        TT_CUDA(cudaMemcpyAsync(op->cores[k], narrowed[k].data(), narrowed[k].size() * sizeof(T),
                                cudaMemcpyHostToDevice, c->stream));
        op->nz_count[k] = (long)vals[k].size();
        op->nz_ptr[k] = (const int*)p;
        TT_CUDA(cudaMemcpyAsync(p, ptr[k].data(), ptr[k].size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        p += al(ptr[k].size() * sizeof(int));
        op->nz_j[k] = (const int*)p;
        if (!js[k].empty())
            TT_CUDA(cudaMemcpyAsync(p, js[k].data(), js[k].size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        p += al(std::max<size_t>(1, js[k].size()) * sizeof(int));
        op->nz_val[k] = p;
        if (!vals[k].empty())
            TT_CUDA(cudaMemcpyAsync(p, vals[k].data(), vals[k].size() * sizeof(T), cudaMemcpyHostToDevice,
                                    c->stream));
        p += al(std::max<size_t>(1, vals[k].size()) * sizeof(T));
    }
    c->sync();  // the host vectors are released on return
}

void upload_cores(tt_operator* op, const double* const* host) {
    if (op->dtype == TT_DTYPE_F64) upload_t<double>(op, host);
    else upload_t<float>(op, host);
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
        if ((long)op->R[k] * op->m[k] * op->R[k + 1] > INT32_MAX)
            throw_status(TT_ERR_ARG, "tt_matvec: operator core with more than 2^31 - 1 (a, i, b) triples");
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
        const long nnz = op->nz_count[k];
        if (ctx->prec == TT_FP64)
            matvec_core<double>(*ctx, op->nz_ptr[k], op->nz_j[k], (const double*)op->nz_val[k], nnz,
                                (const double*)x->cores[k], (double*)y->cores[k], op->R[k], x->r[k], op->m[k],
                                op->n[k], op->R[k + 1], x->r[k + 1]);
        else
            matvec_core<float>(*ctx, op->nz_ptr[k], op->nz_j[k], (const float*)op->nz_val[k], nnz,
                               (const float*)x->cores[k], (float*)y->cores[k], op->R[k], x->r[k], op->m[k],
                               op->n[k], op->R[k + 1], x->r[k + 1]);
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
