// C ABI: contexts, tensors, TT sum / scale / dot / norm (Section 2).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "api_common.h"

namespace ttgb {

static thread_local std::string g_last_error;

void set_last_error(const std::string& s) { g_last_error = s; }

[[noreturn]] void throw_status(tt_status s, const std::string& msg) { throw Error{s, msg}; }

[[noreturn]] void throw_cuda(cudaError_t e, const char* what, const char* file, int line) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e) + " at " + file + ":" + std::to_string(line);
    if (e == cudaErrorMemoryAllocation) throw Error{TT_ERR_OOM, m};
    throw Error{TT_ERR_CUDA, m};
}

void* Ctx::alloc(size_t bytes) {
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~size_t(255);
    Ctx& a = root ? *root : *this;  // lanes draw on their root's budget
    {
        std::lock_guard<std::mutex> lk(a.acct_mu);
        if (a.budget && a.stats.bytes_in_use + bytes > a.budget)
            throw_status(TT_ERR_OOM, "HBM budget exceeded (" + std::to_string(a.stats.bytes_in_use + bytes) +
                                         " > " + std::to_string(a.budget) + " bytes)");
        a.stats.bytes_in_use += bytes;
        a.stats.peak_bytes = std::max<uint64_t>(a.stats.peak_bytes, a.stats.bytes_in_use);
    }
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes, stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        std::lock_guard<std::mutex> lk(a.acct_mu);
        a.stats.bytes_in_use -= std::min<uint64_t>(a.stats.bytes_in_use, bytes);
        throw_status(TT_ERR_OOM, std::string("device allocation failed: ") + cudaGetErrorString(e));
    }
    return p;
}

void Ctx::release(void* p, size_t bytes) {
    if (!p) return;
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~size_t(255);
    cudaFreeAsync(p, stream);
    Ctx& a = root ? *root : *this;
    std::lock_guard<std::mutex> lk(a.acct_mu);
    a.stats.bytes_in_use -= std::min<uint64_t>(a.stats.bytes_in_use, bytes);
}

void Ctx::sync() {
    stats.host_syncs++;
    TT_CUDA(cudaStreamSynchronize(stream));
}

int Ctx::family(const char* name) {
    for (size_t i = 0; i < fam_names.size(); ++i)
        if (fam_names[i] == name) return (int)i;
    fam_names.push_back(name);
    return (int)fam_names.size() - 1;
}

cudaEvent_t Ctx::event() {
    if (!ev_pool.empty()) {
        cudaEvent_t e = ev_pool.back();
        ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    TT_CUDA(cudaEventCreate(&e));
    return e;
}

cudaStream_t Ctx::copies() {
    if (!copy_stream) TT_CUDA(cudaStreamCreateWithFlags(&copy_stream, cudaStreamNonBlocking));
    return copy_stream;
}

cudaStream_t Ctx::crit() {
    if (!crit_stream) {
        int least = 0, greatest = 0;
        TT_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        TT_CUDA(cudaStreamCreateWithPriority(&crit_stream, cudaStreamNonBlocking, greatest));
    }
    return crit_stream;
}

cudaStream_t Ctx::crit2() {
    if (!crit2_stream) {
        int least = 0, greatest = 0;
        TT_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        TT_CUDA(cudaStreamCreateWithPriority(&crit2_stream, cudaStreamNonBlocking, greatest));
    }
    return crit2_stream;
}

cudaStream_t Ctx::side() {
    if (!side_stream) TT_CUDA(cudaStreamCreateWithFlags(&side_stream, cudaStreamNonBlocking));
    return side_stream;
}

cudaStream_t Ctx::tail() {
    if (!tail_stream) TT_CUDA(cudaStreamCreateWithFlags(&tail_stream, cudaStreamNonBlocking));
    return tail_stream;
}

void* Ctx::pinned_words() {
    if (!host_words) TT_CUDA(cudaHostAlloc(&host_words, kHostWords, cudaHostAllocDefault));
    return host_words;
}

Ctx::~Ctx() {
    if (copy_stream) {
        cudaStreamSynchronize(copy_stream);
        cudaStreamDestroy(copy_stream);
    }
    for (cudaStream_t* s : {&crit_stream, &crit2_stream, &side_stream, &tail_stream})
        if (*s) {
            cudaStreamSynchronize(*s);
            cudaStreamDestroy(*s);
        }
    if (host_words) cudaFreeHost(host_words);
    for (Ctx* l : lanes) {
        cudaStreamSynchronize(l->stream);
        delete static_cast<tt_ctx*>(l);  // lanes are allocated as tt_ctx
    }
    if (owns_stream && stream) cudaStreamDestroy(stream);
    for (auto& r : recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : ev_pool) cudaEventDestroy(e);
    if (tc_err) cudaFree(tc_err);
}

void check_tc_error(Ctx& c) {
    int h = 0;
    TT_CUDA(cudaMemcpyAsync(&h, c.tc_err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    if (h) {
        TT_CUDA(cudaMemsetAsync(c.tc_err, 0, sizeof(int), c.stream));
        throw_status(TT_ERR_TIMEOUT, "a bounded wait inside a tensor-core kernel ran out");
    }
}

ProfScope::ProfScope(Ctx& ctx, const char* name, double fl, double by) : c(ctx), flops(fl), bytes(by) {
    // only the outermost scope records: launches made inside another
    // instrumented call (the GEMMs of the blocked Cholesky) count for it
    if (c.prof_nest++ > 0 || !c.prof) return;
    if (!c.prof_only.empty() && c.prof_only != name) return;
    fam = c.family(name);
    a = c.event();
    TT_CUDA(cudaEventRecord(a, c.stream));
}

ProfScope::~ProfScope() {
    c.prof_nest--;
    if (!a) return;
    cudaEvent_t b = c.event();
    cudaEventRecord(b, c.stream);
    c.recs.push_back(ProfRec{fam, flops, bytes, a, b});
}

size_t dtype_size(tt_dtype t) { return t == TT_DTYPE_F64 ? 8 : 4; }

tt_dtype storage_of(tt_precision p) { return p == TT_FP64 ? TT_DTYPE_F64 : TT_DTYPE_F32; }

void validate_shape(int d, const int* n, const int* r) {
    if (d < 1 || !n || !r) throw_status(TT_ERR_ARG, "d < 1 or NULL shape");
    if (r[0] != 1 || r[d] != 1) throw_status(TT_ERR_ARG, "r_0 and r_d must be 1");
    for (int k = 0; k < d; ++k) {
        if (n[k] < 1) throw_status(TT_ERR_ARG, "mode size < 1");
        if (r[k + 1] < 1) throw_status(TT_ERR_ARG, "rank < 1");
    }
}

tt_tensor* new_tensor(tt_ctx* ctx, int d, const int* n, const int* r) {
    validate_shape(d, n, r);
    tt_tensor* t = new tt_tensor();
    t->ctx = ctx;
    t->d = d;
    t->n.assign(n, n + d);
    t->r.assign(r, r + d + 1);
    t->dtype = storage_of(ctx->prec);
    t->cores.assign(d, nullptr);
    size_t es = dtype_size(t->dtype), off = 0;
    std::vector<size_t> offs(d);
    for (int k = 0; k < d; ++k) {
        offs[k] = off;
        off += ((size_t)r[k] * n[k] * r[k + 1] * es + 255) & ~size_t(255);
    }
    try {
        t->block = ctx->alloc(off);
    } catch (...) {
        delete t;
        throw;
    }
    t->bytes = off;
    t->owned = true;
    for (int k = 0; k < d; ++k) t->cores[k] = (char*)t->block + offs[k];
    ctx->refs++;
    return t;
}

void drop_ctx_ref(tt_ctx* c) {
    if (--c->refs == 0) {
        cudaStreamSynchronize(c->stream);
        delete c;
    }
}

void free_tensor(tt_tensor* t) {
    if (!t) return;
    tt_ctx* c = t->ctx;
    if (t->owned && t->block) c->release(t->block, t->bytes);
    delete t;
    drop_ctx_ref(c);
}

void check_same_modes(const tt_tensor* a, const tt_tensor* b) {
    if (a->d != b->d) throw_status(TT_ERR_SHAPE, "orders differ");
    for (int k = 0; k < a->d; ++k)
        if (a->n[k] != b->n[k]) throw_status(TT_ERR_SHAPE, "mode sizes differ");
}

void check_tensor(tt_ctx* ctx, const tt_tensor* x) {
    if (!x) throw_status(TT_ERR_ARG, "NULL tensor");
    // a lane may read its root's tensors (the caller orders the streams)
    const Ctx* hx = x->ctx->root ? x->ctx->root : static_cast<const Ctx*>(x->ctx);
    const Ctx* hc = ctx->root ? ctx->root : static_cast<const Ctx*>(ctx);
    if (hx != hc) throw_status(TT_ERR_ARG, "tensor belongs to another context");
}

tt_tensor* copy_tensor(tt_ctx* ctx, const tt_tensor* x) {
    tt_tensor* y = new_tensor(ctx, x->d, x->n.data(), x->r.data());
    size_t es = dtype_size(x->dtype);
    for (int k = 0; k < x->d; ++k)
        TT_CUDA(cudaMemcpyAsync(y->cores[k], x->cores[k], es * x->core_elems(k), cudaMemcpyDeviceToDevice,
                                ctx->stream));
    y->norm_hint = x->norm_hint;
    return y;
}

// ---------------------------------------------------------------- TT sum
template <class T>
tt_tensor* add_impl(tt_ctx* ctx, int m, const double* alpha, const tt_tensor* const* x) {
    const tt_tensor* x0 = x[0];
    const int d = x0->d;
    std::vector<int> r(d + 1, 0);
    r[0] = 1;
    r[d] = 1;
    for (int k = 1; k < d; ++k)
        for (int j = 0; j < m; ++j) r[k] += x[j]->r[k];
    if (d == 1) {
        // linear combination of the single cores (1 x n x 1)
        int one[2] = {1, 1};
        tt_tensor* y = new_tensor(ctx, 1, x0->n.data(), one);
        TT_CUDA(cudaMemsetAsync(y->cores[0], 0, sizeof(T) * x0->n[0], ctx->stream));
        for (int j = 0; j < m; ++j) axpy<T>(*ctx, x0->n[0], alpha[j], (const T*)x[j]->cores[0], (T*)y->cores[0]);
        return y;
    }
    tt_tensor* y = new_tensor(ctx, d, x0->n.data(), r.data());
    for (int k = 0; k < d; ++k) {
        const int n = x0->n[k];
        const long RB = r[k + 1];
        if (k > 0 && k < d - 1)
            TT_CUDA(cudaMemsetAsync(y->cores[k], 0, sizeof(T) * y->core_elems(k), ctx->stream));
        long oa = 0, ob = 0;
        for (int j0 = 0; j0 < m; j0 += 64) {
            BlockList list;
            list.count = std::min(64, m - j0);
            int ma = 0, mb = 0;
            for (int t = 0; t < list.count; ++t) {
                const int j = j0 + t;
                const int a = x[j]->r[k], b = x[j]->r[k + 1];
                const long oaa = (k == 0) ? 0 : oa;
                const long obb = (k == d - 1) ? 0 : ob;
                list.blk[t] = BlockDesc{x[j]->cores[k], oaa * n * RB + obb, a, b, k == 0 ? alpha[j] : 1.0};
                oa += a;
                ob += b;
                ma = std::max(ma, a);
                mb = std::max(mb, b);
            }
            scatter_blocks<T>(*ctx, list, n, RB, (long)n * RB, (T*)y->cores[k], ma, mb);
        }
    }
    return y;
}

tt_tensor* tt_add_internal(tt_ctx* ctx, int m, const double* alpha, const tt_tensor* const* x) {
    if (m < 1 || !alpha || !x) throw_status(TT_ERR_ARG, "tt_add: m < 1 or NULL");
    for (int j = 0; j < m; ++j) {
        check_tensor(ctx, x[j]);
        check_same_modes(x[0], x[j]);
        if (!isfinite(alpha[j])) throw_status(TT_ERR_ARG, "tt_add: non-finite coefficient");
    }
    if (ctx->prec == TT_FP64) return add_impl<double>(ctx, m, alpha, x);
    return add_impl<float>(ctx, m, alpha, x);
}

tt_tensor* scale_internal(tt_ctx* ctx, const tt_tensor* x, double alpha) {
    tt_tensor* y = copy_tensor(ctx, x);
    const int k = x->d - 1;
    if (ctx->prec == TT_FP64) scale_inplace<double>(*ctx, y->core_elems(k), (double*)y->cores[k], alpha);
    else scale_inplace<float>(*ctx, y->core_elems(k), (float*)y->cores[k], alpha);
    y->norm_hint = x->norm_hint >= 0 ? x->norm_hint * fabs(alpha) : -1.0;
    return y;
}

// ---------------------------------------------------------------- TT dot
// W_0 = 1; V = W_{k-1} Y_k^R (r_x x n r_y'); W_k = (X_k^L)^T V^L.
template <class T>
void dot_chain(tt_ctx* ctx, const tt_tensor* x, const tt_tensor* y, T* wsA, T* wsV, T* out_dev) {
    const int d = x->d;
    T* W = wsA;  // r_x x r_y
    // W_0 = 1
    fill_identity<T>(*ctx, 1, W, 1);
    for (int k = 0; k < d; ++k) {
        const int n = x->n[k];
        const int rx = x->r[k], rx2 = x->r[k + 1], ry = y->r[k], ry2 = y->r[k + 1];
        // V (rx x n*ry2) = W (rx x ry) * Y^R (ry x n*ry2)
        gemm<T>(*ctx, false, false, rx, n * ry2, ry, T(1), W, ry, (const T*)y->cores[k], (long)n * ry2, T(0), wsV,
                (long)n * ry2);
        // W' (rx2 x ry2) = X^L^T (rx2 x rx*n) * V^L (rx*n x ry2)
        T* Wn = (k == d - 1) ? out_dev : W;
        gemm<T>(*ctx, true, false, rx2, ry2, rx * n, T(1), (const T*)x->cores[k], rx2, wsV, ry2, T(0), Wn, ry2);
    }
}

size_t dot_ws_elems(const tt_tensor* x, const tt_tensor* y, size_t* wA) {
    size_t a = 1, v = 1;
    for (int k = 0; k < x->d; ++k) {
        a = std::max(a, (size_t)x->r[k + 1] * y->r[k + 1]);
        a = std::max(a, (size_t)x->r[k] * y->r[k]);
        v = std::max(v, (size_t)x->r[k] * x->n[k] * y->r[k + 1]);
    }
    *wA = a;
    return v;
}

template <class T>
void dot_many_impl(tt_ctx* ctx, const tt_tensor* x, int count, const tt_tensor* const* y, double* out) {
    size_t wa = 1, wv = 1;
    for (int j = 0; j < count; ++j) {
        size_t a;
        wv = std::max(wv, dot_ws_elems(x, y[j], &a));
        wa = std::max(wa, a);
    }
    const size_t bytes = sizeof(T) * (wa + wv + count + 2) + 512;
    char* ws = (char*)ctx->alloc(bytes);
    T* A = (T*)ws;
    T* V = A + wa;
    T* res = V + wv;
    for (int j = 0; j < count; ++j) dot_chain<T>(ctx, x, y[j], A, V, res + j);
    std::vector<T> h(count);
    TT_CUDA(cudaMemcpyAsync(h.data(), res, sizeof(T) * count, cudaMemcpyDeviceToHost, ctx->stream));
    ctx->sync();
    ctx->release(ws, bytes);
    for (int j = 0; j < count; ++j) out[j] = (double)h[j];
}

// FP32-stored cores, FP64 accumulation: the cores are widened to FP64 in a
// workspace and contracted with FP64 GEMMs, so the scalars that drive the
// orthogonalization schemes (projections, norms) carry no FP32 summation error.
void dot_many_f32_acc64(tt_ctx* ctx, const tt_tensor* x, int count, const tt_tensor* const* y, double* out) {
    size_t wa = 1, wv = 1, xe = 0, ye = 0;
    for (int k = 0; k < x->d; ++k) xe += x->core_elems(k);
    for (int j = 0; j < count; ++j) {
        size_t a, e = 0;
        wv = std::max(wv, dot_ws_elems(x, y[j], &a));
        wa = std::max(wa, a);
        for (int k = 0; k < y[j]->d; ++k) e += y[j]->core_elems(k);
        ye = std::max(ye, e);
    }
    const size_t bytes = sizeof(double) * (wa + wv + count + 2 + xe + ye) + 1024;
    char* ws = (char*)ctx->alloc(bytes);
    double* A = (double*)ws;
    double* V = A + wa;
    double* res = V + wv;
    double* xc = res + count + 2;
    double* yc = xc + xe;
    tt_tensor xd = *x, yd;
    size_t off = 0;
    for (int k = 0; k < x->d; ++k) {
        convert<float, double>(*ctx, (long)x->core_elems(k), (const float*)x->cores[k], xc + off);
        xd.cores[k] = xc + off;
        off += x->core_elems(k);
    }
    for (int j = 0; j < count; ++j) {
        yd = *y[j];
        off = 0;
        for (int k = 0; k < y[j]->d; ++k) {
            convert<float, double>(*ctx, (long)y[j]->core_elems(k), (const float*)y[j]->cores[k], yc + off);
            yd.cores[k] = yc + off;
            off += y[j]->core_elems(k);
        }
        dot_chain<double>(ctx, &xd, &yd, A, V, res + j);
    }
    std::vector<double> h(count);
    TT_CUDA(cudaMemcpyAsync(h.data(), res, sizeof(double) * count, cudaMemcpyDeviceToHost, ctx->stream));
    ctx->sync();
    ctx->release(ws, bytes);
    for (int j = 0; j < count; ++j) out[j] = h[j];
}

// ---------------------------------------------------------------- stacked dots
// <x, y_j> for all j at once: the contractions of all pairs advance
// together, core by core.  W (rx x S, FP64) holds the pairs' W_j side by
// side (S = sum_j ry_j).  Step A: V (rx n x S', storage type) with
// V[(a n + i), off'_j + q] = sum_b W[a, off_j + b] Y_j(b, i, q) (sums of ry_j
// terms in the storage type, one small product per pair; FP64 sums in the
// fallback for very large ranks).  Step B: W' = X_k^L^T V, one GEMM over all pairs, so X's
// cores are read once for all pairs (the pair-by-pair chains read them once
// per pair, in two small launches per core each).  FP64 storage: one FP64
// GEMM.  FP32 storage: FP32 GEMMs over chunks of kDotChunk rows of X^L whose
// partial products are summed in FP64, so each coefficient carries FP32
// products and FP32 sums of at most kDotChunk terms (about 1e-6 of the sum
// of the terms' magnitudes).
namespace {
constexpr int kDotChunk = 256;

template <class T>
struct PairCols {
    const T* y;     // core k of y_j
    int ry, ry2;    // its ranks
    int off, off2;  // its column offsets in W and V
};

template <class T>
__global__ void stack_a_kernel(const double* __restrict__ W, int S, const PairCols<T>* __restrict__ pairs,
                               int npairs, int rx, int n, int S2, T* __restrict__ V) {
    const long total = (long)rx * n * S2;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int col = (int)(t % S2);
        const long row = t / S2;
        const int i = (int)(row % n), a = (int)(row / n);
        int lo = 0, hi = npairs - 1;  // the pair whose columns hold col
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pairs[mid].off2 <= col) lo = mid;
            else hi = mid - 1;
        }
        const PairCols<T> pc = pairs[lo];
        const int q = col - pc.off2;
        const double* w = W + (long)a * S + pc.off;
        const T* y = pc.y + (long)i * pc.ry2 + q;  // Y(b, i, q) at y[b n ry2]
        double acc = 0.0;
        for (int b = 0; b < pc.ry; ++b) acc += w[b] * (double)y[(long)b * n * pc.ry2];
        V[t] = (T)acc;
    }
}

// Step A as one small product per pair, V_j = W_j Y_j (rx x n ry2_j): block
// (x, y) takes 128 columns (i, q) of pair y, thread c one column, and runs
// over the rows a in chunks of kStackRows with W_j's chunk in shared memory
// (read by broadcast) and the column of Y_j read once per chunk, so Y_j is
// read rx / kStackRows times instead of rx times.  Sums in the storage type:
// FP32 storage sums the ry_j terms in FP32 (the FP32 products of step B sum
// kDotChunk terms in FP32 as well); FP64 storage in FP64.
constexpr int kStackRows = 16;

template <class T>
__global__ void __launch_bounds__(128) stack_a_tiled_kernel(const double* __restrict__ W, int S,
                                                            const PairCols<T>* __restrict__ pairs, int rx, int n,
                                                            int S2, T* __restrict__ V) {
    extern __shared__ __align__(16) unsigned char stack_sm[];
    T* Ws = reinterpret_cast<T*>(stack_sm);  // kStackRows x ry, row-major
    const PairCols<T> pc = pairs[blockIdx.y];
    const int ncols = n * pc.ry2;
    if ((long)blockIdx.x * blockDim.x >= ncols) return;  // the whole block is past this pair's columns
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = c < ncols;
    const int i = live ? c / pc.ry2 : 0;
    const int q = live ? c - i * pc.ry2 : 0;
    const T* y = pc.y + (long)i * pc.ry2 + q;  // Y(b, i, q) at y[b n ry2]
    const long ystride = (long)n * pc.ry2;
    for (int a0 = 0; a0 < rx; a0 += kStackRows) {
        const int na = min(kStackRows, rx - a0);
        __syncthreads();  // the previous chunk's W is no longer read
        for (int e = threadIdx.x; e < kStackRows * pc.ry; e += blockDim.x) {
            const int aa = e / pc.ry, b = e - aa * pc.ry;
            Ws[e] = aa < na ? (T)W[(long)(a0 + aa) * S + pc.off + b] : T(0);
        }
        __syncthreads();
        if (!live) continue;
        T acc[kStackRows];
#pragma unroll
        for (int aa = 0; aa < kStackRows; ++aa) acc[aa] = T(0);
        for (int b = 0; b < pc.ry; ++b) {
            const T yb = y[(long)b * ystride];
#pragma unroll
            for (int aa = 0; aa < kStackRows; ++aa) acc[aa] = fma(Ws[aa * pc.ry + b], yb, acc[aa]);
        }
#pragma unroll
        for (int aa = 0; aa < kStackRows; ++aa)
            if (aa < na) V[((long)(a0 + aa) * n + i) * S2 + pc.off2 + q] = acc[aa];
    }
}

template <class T>
__global__ void sum_chunks_kernel(const T* __restrict__ P, long chunk_elems, int nchunks, double* __restrict__ out) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < chunk_elems; e += (long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int c = 0; c < nchunks; ++c) acc += (double)P[(long)c * chunk_elems + e];
        out[e] = acc;
    }
}

unsigned grid_of(const Ctx& c, long total, int threads) {
    const long want = (total + threads - 1) / threads;
    return (unsigned)std::max(1L, std::min(want, (long)std::max(1, c.sm_count) * 8));
}
}  // namespace

template <class T>
void dot_many_stacked(tt_ctx* ctx, const tt_tensor* x, int count, const tt_tensor* const* y, double* out) {
    const bool f32 = sizeof(T) == 4;
    const int d = x->d;
    size_t wmax = 1, vmax = 1, pmax = 1;
    for (int k = 0; k < d; ++k) {
        long S = 0, S2 = 0;
        for (int j = 0; j < count; ++j) {
            S += y[j]->r[k];
            S2 += y[j]->r[k + 1];
        }
        if (S2 > (1L << 24) || S > (1L << 24)) throw_status(TT_ERR_ARG, "tt_dot_many: too many stacked columns");
        const long K = (long)x->r[k] * x->n[k];
        const long nch = f32 ? (K + kDotChunk - 1) / kDotChunk : 1;
        wmax = std::max(wmax, (size_t)x->r[k] * S);
        wmax = std::max(wmax, (size_t)x->r[k + 1] * S2);
        vmax = std::max(vmax, (size_t)K * S2);
        pmax = std::max(pmax, (size_t)nch * x->r[k + 1] * S2);
    }
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t bytes =
        2 * al(wmax * 8) + al(vmax * sizeof(T)) + al(pmax * sizeof(T)) + al((size_t)count * sizeof(PairCols<T>)) + 512;
    char* ws = (char*)ctx->alloc(bytes);
    struct Rel {
        tt_ctx* c; void* p; size_t b;
        ~Rel() { c->release(p, b); }
    } rel{ctx, ws, bytes};
    char* p = ws;
    double* W = (double*)p; p += al(wmax * 8);
    double* W2 = (double*)p; p += al(wmax * 8);
    T* V = (T*)p; p += al(vmax * sizeof(T));
    T* P = (T*)p; p += al(pmax * sizeof(T));
    PairCols<T>* dpairs = (PairCols<T>*)p;
    std::vector<PairCols<T>> hp(count);
    {
        // W_0 = 1 for every pair (r_0 = 1); a pageable source is staged
        // before the call returns
        std::vector<double> ones(count, 1.0);
        TT_CUDA(cudaMemcpyAsync(W, ones.data(), count * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    }
    for (int k = 0; k < d; ++k) {
        const int rx = x->r[k], rx2 = x->r[k + 1], n = x->n[k];
        int S = 0, S2 = 0;
        for (int j = 0; j < count; ++j) {
            hp[j] = PairCols<T>{(const T*)y[j]->cores[k], y[j]->r[k], y[j]->r[k + 1], S, S2};
            S += y[j]->r[k];
            S2 += y[j]->r[k + 1];
        }
        // pageable source: the copy is staged before the call returns, and
        // it lands after the previous core's step A (stream order)
        TT_CUDA(cudaMemcpyAsync(dpairs, hp.data(), count * sizeof(PairCols<T>), cudaMemcpyHostToDevice, ctx->stream));
        const long K = (long)rx * n;
        {
            int rymax = 1, colmax = 1;
            for (int j = 0; j < count; ++j) {
                rymax = std::max(rymax, hp[j].ry);
                colmax = std::max(colmax, n * hp[j].ry2);
            }
            const size_t smem = (size_t)kStackRows * rymax * sizeof(T);
            ProfScope ps(*ctx, "dot_stack", 2.0 * (double)K * S2 * 4.0, sizeof(T) * (double)K * S2);
            if (smem <= 48 * 1024 && count <= 65535)
                stack_a_tiled_kernel<T><<<dim3((unsigned)((colmax + 127) / 128), (unsigned)count), 128, smem,
                                          ctx->stream>>>(W, S, dpairs, rx, n, S2, V);
            else
                stack_a_kernel<T><<<grid_of(*ctx, K * S2, 256), 256, 0, ctx->stream>>>(W, S, dpairs, count, rx, n, S2,
                                                                                      V);
            TT_LAUNCHED(*ctx);
        }
        const T* X = (const T*)x->cores[k];
        const long ce = (long)rx2 * S2;
        int nch = 1;
        if (f32) {
            // W' (rx2 x S2) = X^L^T V in chunks of K, FP64 sum of the chunks
            const long nfull = K / kDotChunk, rem = K - nfull * kDotChunk;
            if (nfull > 0)
                gemm<T>(*ctx, true, false, rx2, S2, kDotChunk, T(1), X, rx2, V, S2, T(0), P, S2, (int)nfull,
                        (long)kDotChunk * rx2, (long)kDotChunk * S2, ce);
            if (rem > 0)
                gemm<T>(*ctx, true, false, rx2, S2, (int)rem, T(1), X + nfull * kDotChunk * rx2, rx2,
                        V + nfull * kDotChunk * S2, S2, T(0), P + nfull * ce, S2);
            nch = (int)(nfull + (rem > 0 ? 1 : 0));
        } else {
            gemm<T>(*ctx, true, false, rx2, S2, (int)K, T(1), X, rx2, V, S2, T(0), P, S2);
        }
        sum_chunks_kernel<T><<<grid_of(*ctx, ce, 256), 256, 0, ctx->stream>>>(P, ce, nch, W2);
        TT_LAUNCHED(*ctx);
        std::swap(W, W2);
    }
    std::vector<double> h(count);
    TT_CUDA(cudaMemcpyAsync(h.data(), W, sizeof(double) * count, cudaMemcpyDeviceToHost, ctx->stream));
    ctx->sync();
    for (int j = 0; j < count; ++j) out[j] = h[j];
}

void dot_many_internal(tt_ctx* ctx, const tt_tensor* x, int count, const tt_tensor* const* y, double* out,
                       bool stacked) {
    check_tensor(ctx, x);
    if (count < 0 || (count > 0 && (!y || !out))) throw_status(TT_ERR_ARG, "tt_dot_many: bad arguments");
    for (int j = 0; j < count; ++j) {
        check_tensor(ctx, y[j]);
        check_same_modes(x, y[j]);
    }
    if (count == 0) return;
    if (stacked && count >= 2) {
        if (ctx->prec == TT_FP64) dot_many_stacked<double>(ctx, x, count, y, out);
        else dot_many_stacked<float>(ctx, x, count, y, out);
    } else if (ctx->prec == TT_FP64) {
        dot_many_impl<double>(ctx, x, count, y, out);
    } else {
        dot_many_f32_acc64(ctx, x, count, y, out);  // FP64 accumulation throughout
    }
}

}  // namespace ttgb

using namespace ttgb;

// ================================================================ C ABI
extern "C" {

tt_status tt_ctx_create(tt_ctx** out, int device, tt_precision prec, void* stream, size_t hbm_budget) {
    TT_API_BEGIN
    if (!out) throw_status(TT_ERR_ARG, "NULL ctx out");
    *out = nullptr;
    if (prec != TT_FP64 && prec != TT_MIXED_TF32 && prec != TT_FP32) throw_status(TT_ERR_ARG, "bad precision");
    int ndev = 0;
    TT_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) throw_status(TT_ERR_ARG, "bad device");
    TT_CUDA(cudaSetDevice(device));
    cudaDeviceProp prop;
    TT_CUDA(cudaGetDeviceProperties(&prop, device));
    if (prop.major != 10) throw_status(TT_ERR_CUDA, "device is not a Blackwell (sm_10x) GPU");
    tt_ctx* c = new tt_ctx();
    c->device = device;
    c->prec = prec;
    c->stream = (cudaStream_t)stream;
    c->budget = hbm_budget;
    c->sm_count = prop.multiProcessorCount;
    // TTGB_NO_TENSOR_CORES=1 keeps TT_MIXED_TF32 contexts on the CUDA-core Gram
    const char* no_tc = getenv("TTGB_NO_TENSOR_CORES");
    if (no_tc && no_tc[0] == '1') c->use_tc = false;
    // TTGB_TC_GEMM=3 moves the core-producing GEMMs onto the tensor cores
    // (three-part split, 6 products); =2 the two-part split (3 products,
    // ~2^-22 per product); unset or 0 keeps them on CUDA cores
    const char* tg = getenv("TTGB_TC_GEMM");
    if (tg && tg[0] == '3') c->use_tc_gemm = true;
    // =a: only the absorbs (three-part split) on the tensor cores
    if (tg && tg[0] == 'a') c->use_tc_absorb = true;
    if (tg && tg[0] == '2') {
        c->use_tc_gemm = true;
        c->tc_gemm_split = 2;
    }
    // TTGB_CHOL_NB fixes the block size of the Cholesky factorizations (a
    // multiple of 32; 0 or unset: the per-order table)
    const char* nb = getenv("TTGB_CHOL_NB");
    if (nb) c->chol_nb = std::max(0, atoi(nb));
    // TTGB_COLGRAM_STAGES=3 keeps three raw staging stages in the tensor-core
    // column Gram (default five)
    const char* cg = getenv("TTGB_COLGRAM_STAGES");
    if (cg && cg[0] == '3') c->colgram_stages = 3;
    // TTGB_SERIES_PASS=0 keeps the Cholesky factorization for every second
    // Cholesky QR pass (no series pass); =retry treats every series pass as
    // invalid, so each rounding is redone with Cholesky passes (exercises
    // the retry path); =noskip keeps every second pass
    const char* sp = getenv("TTGB_SERIES_PASS");
    if (sp && sp[0] == '0') c->use_series = false;
    if (sp && sp[0] == 'r') c->series_force_retry = true;
    // =noskip: every second pass runs (no first pass is kept alone)
    if (sp && sp[0] == 'n') c->series_no_skip = true;
    // TTGB_PIPELINE=0 runs the sweeps of TT-round on the context's stream
    // alone (no speculative overlap)
    const char* pl = getenv("TTGB_PIPELINE");
    if (pl && pl[0] == '0') c->pipeline = false;
    // TTGB_LANE_PIPELINE=1: the lanes of batched rounding and of the server
    // pipeline their sweeps as well (with the extra workspace in their
    // footprints)
    const char* lp = getenv("TTGB_LANE_PIPELINE");
    if (lp && lp[0] == '1') c->lane_pipeline = true;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    if (cudaMalloc(&c->tc_err, sizeof(int)) != cudaSuccess || cudaMemset(c->tc_err, 0, sizeof(int)) != cudaSuccess) {
        delete c;
        throw_status(TT_ERR_CUDA, "could not allocate the device status word");
    }
    *out = c;
    TT_API_END
}

void tt_ctx_destroy(tt_ctx* ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    drop_ctx_ref(ctx);  // deleted now, or when its last tensor is freed
}

tt_status tt_ctx_get_stats(const tt_ctx* ctx, tt_stats* out) {
    if (!ctx || !out) return TT_ERR_ARG;
    *out = ctx->stats;
    return TT_OK;
}

void tt_ctx_reset_stats(tt_ctx* ctx) {
    if (!ctx) return;
    uint64_t in_use = ctx->stats.bytes_in_use;
    ctx->stats = tt_stats{};
    ctx->stats.bytes_in_use = in_use;
    ctx->stats.peak_bytes = in_use;
}

tt_precision tt_ctx_precision(const tt_ctx* ctx) { return ctx ? ctx->prec : TT_FP64; }

tt_status tt_ctx_set_profiling(tt_ctx* ctx, int on) {
    if (!ctx) return TT_ERR_ARG;
    ctx->prof = on != 0;
    return TT_OK;
}

tt_status tt_ctx_set_pipeline(tt_ctx* ctx, int on) {
    if (!ctx) return TT_ERR_ARG;
    ctx->pipeline = on != 0;
    return TT_OK;
}

tt_status tt_ctx_set_tc_wait_limit(tt_ctx* ctx, long long cycles) {
    if (!ctx || cycles < 0) return TT_ERR_ARG;
    ctx->tc_wait_limit = cycles;
    return TT_OK;
}

tt_status tt_ctx_set_profiling_family(tt_ctx* ctx, const char* family) {
    if (!ctx) return TT_ERR_ARG;
    ctx->prof_only = family ? family : "";
    return TT_OK;
}

void tt_ctx_reset_profile(tt_ctx* ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto& r : ctx->recs) {
        ctx->ev_pool.push_back(r.a);
        ctx->ev_pool.push_back(r.b);
    }
    ctx->recs.clear();
}

tt_status tt_ctx_get_profile(tt_ctx* ctx, tt_kernel_profile* out, int max_entries, int* n_entries) {
    TT_API_BEGIN
    if (!ctx || !n_entries || (max_entries > 0 && !out)) throw_status(TT_ERR_ARG, "bad arguments");
    ctx->sync();
    std::vector<tt_kernel_profile> agg(ctx->fam_names.size());
    for (size_t i = 0; i < agg.size(); ++i) {
        memset(&agg[i], 0, sizeof(agg[i]));
        strncpy(agg[i].name, ctx->fam_names[i].c_str(), sizeof(agg[i].name) - 1);
    }
    for (auto& r : ctx->recs) {
        float ms = 0.f;
        TT_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        tt_kernel_profile& p = agg[r.fam];
        p.launches++;
        p.total_ms += ms;
        p.flops += r.flops;
        p.bytes += r.bytes;
    }
    int k = 0;
    for (auto& p : agg) {
        if (p.launches == 0) continue;
        if (k < max_entries) out[k] = p;
        ++k;
    }
    *n_entries = k;
    TT_API_END
}

tt_status tt_set_sign_rule(tt_ctx* ctx, tt_sign_rule rule) {
    if (!ctx || (rule != TT_SIGN_STABLE && rule != TT_SIGN_LITERAL)) return TT_ERR_ARG;
    ctx->sign_rule = rule;
    return TT_OK;
}

tt_status tt_tensor_create(tt_ctx* ctx, int d, const int* n, const int* r, const double* const* host_cores,
                           tt_tensor** out) {
    TT_API_BEGIN
    if (!ctx || !out) throw_status(TT_ERR_ARG, "NULL argument");
    *out = nullptr;
    tt_tensor* t = new_tensor(ctx, d, n, r);
    try {
        for (int k = 0; k < d; ++k) {
            const size_t ne = t->core_elems(k);
            if (!host_cores || !host_cores[k]) {
                TT_CUDA(cudaMemsetAsync(t->cores[k], 0, ne * dtype_size(t->dtype), ctx->stream));
            } else if (t->dtype == TT_DTYPE_F64) {
                TT_CUDA(cudaMemcpyAsync(t->cores[k], host_cores[k], ne * 8, cudaMemcpyHostToDevice, ctx->stream));
            } else {
                // FP64 staging on the device, narrowed there (stream-ordered
                // release); the host arrays are read before the call returns
                double* st = (double*)ctx->alloc(ne * 8);
                TT_CUDA(cudaMemcpyAsync(st, host_cores[k], ne * 8, cudaMemcpyHostToDevice, ctx->stream));
                convert<double, float>(*ctx, (long)ne, st, (float*)t->cores[k]);
                ctx->release(st, ne * 8);
            }
        }
        bool pinned = false;
        for (int k = 0; host_cores && k < d && !pinned; ++k) {
            cudaPointerAttributes at;
            pinned = host_cores[k] && cudaPointerGetAttributes(&at, host_cores[k]) == cudaSuccess &&
                     at.type == cudaMemoryTypeHost;
        }
        cudaGetLastError();
        if (pinned) ctx->sync();  // page-locked sources are read asynchronously
    } catch (...) {
        free_tensor(t);
        throw;
    }
    *out = t;
    TT_API_END
}

tt_status tt_tensor_create_storage(tt_ctx* ctx, int d, const int* n, const int* r, const void* const* host_cores,
                                   tt_tensor** out) {
    TT_API_BEGIN
    if (!ctx || !out || !host_cores) throw_status(TT_ERR_ARG, "NULL argument");
    *out = nullptr;
    tt_tensor* t = new_tensor(ctx, d, n, r);
    try {
        for (int k = 0; k < d; ++k) {
            if (!host_cores[k]) throw_status(TT_ERR_ARG, "NULL host core");
            const size_t bytes = t->core_elems(k) * dtype_size(t->dtype);
            TT_CUDA(cudaMemcpyAsync(t->cores[k], host_cores[k], bytes, cudaMemcpyHostToDevice, ctx->stream));
        }
    } catch (...) {
        free_tensor(t);
        throw;
    }
    *out = t;
    TT_API_END
}

tt_status tt_tensor_download_storage(tt_ctx* ctx, const tt_tensor* x, void* const* host_cores) {
    TT_API_BEGIN
    if (!ctx || !host_cores) throw_status(TT_ERR_ARG, "NULL argument");
    check_tensor(ctx, x);
    for (int k = 0; k < x->d; ++k) {
        if (!host_cores[k]) throw_status(TT_ERR_ARG, "NULL host core");
        const size_t bytes = x->core_elems(k) * dtype_size(x->dtype);
        TT_CUDA(cudaMemcpyAsync(host_cores[k], x->cores[k], bytes, cudaMemcpyDeviceToHost, ctx->stream));
    }
    ctx->sync();
    TT_API_END
}

tt_status tt_tensor_wrap_device(tt_ctx* ctx, int d, const int* n, const int* r, void* const* dev_cores, int dtype,
                                tt_tensor** out) {
    TT_API_BEGIN
    if (!ctx || !out || !dev_cores) throw_status(TT_ERR_ARG, "NULL argument");
    *out = nullptr;
    validate_shape(d, n, r);
    if (dtype != (int)storage_of(ctx->prec)) throw_status(TT_ERR_ARG, "dtype differs from the context storage");
    tt_tensor* t = new tt_tensor();
    t->ctx = ctx;
    t->d = d;
    t->n.assign(n, n + d);
    t->r.assign(r, r + d + 1);
    t->dtype = (tt_dtype)dtype;
    t->cores.assign(dev_cores, dev_cores + d);
    for (int k = 0; k < d; ++k)
        if (!t->cores[k]) {
            delete t;
            throw_status(TT_ERR_ARG, "NULL core");
        }
    t->owned = false;
    ctx->refs++;
    *out = t;
    TT_API_END
}

tt_status tt_tensor_shape(const tt_tensor* x, int* d, int* n, int* r) {
    if (!x) return TT_ERR_ARG;
    if (d) *d = x->d;
    if (n) for (int k = 0; k < x->d; ++k) n[k] = x->n[k];
    if (r) for (int k = 0; k <= x->d; ++k) r[k] = x->r[k];
    return TT_OK;
}

tt_status tt_tensor_core_ptr(const tt_tensor* x, int k, void** p) {
    if (!x || !p || k < 0 || k >= x->d) return TT_ERR_ARG;
    *p = x->cores[k];
    return TT_OK;
}

tt_status tt_tensor_download(tt_ctx* ctx, const tt_tensor* x, double* const* host_cores) {
    TT_API_BEGIN
    if (!ctx || !host_cores) throw_status(TT_ERR_ARG, "NULL argument");
    check_tensor(ctx, x);
    for (int k = 0; k < x->d; ++k) {
        if (!host_cores[k]) throw_status(TT_ERR_ARG, "NULL host core");
        const size_t ne = x->core_elems(k);
        if (x->dtype == TT_DTYPE_F64) {
            TT_CUDA(cudaMemcpyAsync(host_cores[k], x->cores[k], ne * 8, cudaMemcpyDeviceToHost, ctx->stream));
        } else {
            double* st = (double*)ctx->alloc(ne * 8);
            convert<float, double>(*ctx, (long)ne, (const float*)x->cores[k], st);
            TT_CUDA(cudaMemcpyAsync(host_cores[k], st, ne * 8, cudaMemcpyDeviceToHost, ctx->stream));
            ctx->release(st, ne * 8);
        }
    }
    ctx->sync();
    TT_API_END
}

void tt_tensor_free(tt_tensor* x) { free_tensor(x); }

tt_status tt_add(tt_ctx* ctx, int m, const double* alpha, const tt_tensor* const* x, tt_tensor** out) {
    TT_API_BEGIN
    if (!ctx || !out) throw_status(TT_ERR_ARG, "NULL argument");
    *out = nullptr;
    *out = tt_add_internal(ctx, m, alpha, x);
    TT_API_END
}

tt_status tt_scale(tt_ctx* ctx, const tt_tensor* x, double alpha, tt_tensor** out) {
    TT_API_BEGIN
    if (!ctx || !out) throw_status(TT_ERR_ARG, "NULL argument");
    *out = nullptr;
    check_tensor(ctx, x);
    if (!isfinite(alpha)) throw_status(TT_ERR_ARG, "non-finite alpha");
    *out = scale_internal(ctx, x, alpha);
    TT_API_END
}

tt_status tt_dot(tt_ctx* ctx, const tt_tensor* x, const tt_tensor* y, double* out) {
    TT_API_BEGIN
    if (!ctx || !out || !y) throw_status(TT_ERR_ARG, "NULL argument");
    const tt_tensor* ys[1] = {y};
    dot_many_internal(ctx, x, 1, ys, out);
    TT_API_END
}

tt_status tt_dot_many(tt_ctx* ctx, const tt_tensor* x, int count, const tt_tensor* const* y, double* out) {
    TT_API_BEGIN
    if (!ctx) throw_status(TT_ERR_ARG, "NULL argument");
    dot_many_internal(ctx, x, count, y, out);
    TT_API_END
}

tt_status tt_gram_f32(tt_ctx* ctx, int n, long K, const float* X, long ldx, float* G, int use_tensor_cores) {
    TT_API_BEGIN
    if (!ctx || !X || !G || n < 1 || K < 1 || ldx < (use_tensor_cores == 2 ? (long)n : K))
        throw_status(TT_ERR_ARG, "bad arguments");
    if (use_tensor_cores == 2) {
        // column Gram: X is K x n row-major (ldx >= n), G = X^T X
        if (!gram_cols_tc_tf32(*ctx, n, K, X, ldx, G)) throw_status(TT_ERR_ARG, "layout not supported by TMA");
        check_tc_error(*ctx);
    } else if (use_tensor_cores) {
        if (!gram_rows_tc_tf32(*ctx, n, K, X, ldx, G)) throw_status(TT_ERR_ARG, "layout not supported by TMA");
        check_tc_error(*ctx);
    } else {
        gram<float, float>(*ctx, true, n, K, X, ldx, G);
        ctx->sync();
    }
    TT_API_END
}

tt_status tt_gemm_f32(tt_ctx* ctx, int trans_b, int M, int N, int K, const float* A, long lda, const float* B,
                      long ldb, float* C, long ldc, int use_tensor_cores) {
    TT_API_BEGIN
    if (!ctx || !A || !B || !C || M < 1 || N < 1 || K < 1) throw_status(TT_ERR_ARG, "bad arguments");
    if (use_tensor_cores) {
        if (use_tensor_cores != 1 && use_tensor_cores != 2) throw_status(TT_ERR_ARG, "use_tensor_cores must be 0, 1 or 2");
        if (!gemm_tc3_tf32(*ctx, trans_b != 0, M, N, K, A, lda, B, ldb, C, ldc, use_tensor_cores == 1 ? 3 : 2))
            throw_status(TT_ERR_ARG, "layout not supported by the tensor-core kernel");
        check_tc_error(*ctx);
    } else {
        gemm<float>(*ctx, false, trans_b != 0, M, N, K, 1.0f, A, lda, B, ldb, 0.0f, C, ldc);
        ctx->sync();
    }
    TT_API_END
}

tt_status tt_cholesky_inverse(tt_ctx* ctx, int n, const void* G, void* L, void* T, double shift_rel,
                              double drop_rel, int* ndrop) {
    TT_API_BEGIN
    if (!ctx || !G || !L || !T || n < 1 || !(shift_rel >= 0.0) || !(drop_rel >= 0.0))
        throw_status(TT_ERR_ARG, "bad arguments");
    CholStatus* st = (CholStatus*)ctx->alloc(sizeof(CholStatus));
    CholStatus h;
    try {
        if (ctx->prec == TT_FP64)
            chol_inv<double, double>(*ctx, n, (const double*)G, (double*)L, (double*)T, shift_rel, drop_rel, st);
        else
            chol_inv<float, float>(*ctx, n, (const float*)G, (float*)L, (float*)T, shift_rel, drop_rel, st);
        TT_CUDA(cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
        ctx->sync();
    } catch (...) {
        ctx->release(st, sizeof(CholStatus));
        throw;
    }
    ctx->release(st, sizeof(CholStatus));
    if (h.nonfinite) throw_status(TT_ERR_NONFINITE, "NaN or Inf in G");
    if (ndrop) *ndrop = h.ndrop;
    TT_API_END
}

const char* tt_status_str(tt_status s) {
    switch (s) {
        case TT_OK: return "TT_OK";
        case TT_ERR_ARG: return "TT_ERR_ARG";
        case TT_ERR_SHAPE: return "TT_ERR_SHAPE";
        case TT_ERR_OOM: return "TT_ERR_OOM";
        case TT_ERR_NOT_SPD: return "TT_ERR_NOT_SPD";
        case TT_ERR_BREAKDOWN: return "TT_ERR_BREAKDOWN";
        case TT_ERR_NONFINITE: return "TT_ERR_NONFINITE";
        case TT_ERR_TIMEOUT: return "TT_ERR_TIMEOUT";
        case TT_ERR_CUDA: return "TT_ERR_CUDA";
        case TT_ERR_CANCELLED: return "TT_ERR_CANCELLED";
    }
    return "TT_ERR_UNKNOWN";
}

const char* tt_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
