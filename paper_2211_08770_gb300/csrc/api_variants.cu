// Variants of TT-rounding beside the Cholesky QR sweeps of api_round.cu:
//
// * Gram-SVD rounding: the left-to-right truncation of TT-round (Section 2)
//   computed from the Gram matrices of the left and right parts of x at each
//   bond, without orthogonalizing the cores.  One right-to-left sweep of
//   contractions gives G_R at every bond; then, bond by bond, the Gram G_L
//   of the current left unfolding, G_L = A A^T and G_R = B B^T (Cholesky
//   with numerically zero pivots dropped), the SVD A^T B = U S V^T, the
//   truncation rank from S, core_k <- core_k A^{-T} U_r and core_{k+1} <-
//   S_r V_r^T B^{-1} core_{k+1}.  GEMMs plus r x r factorizations; the
//   squared condition numbers of the Grams limit the accuracy to about
//   sqrt(r u) ||x||.
// * Randomized rounding (the large-scale variant cited in Section 2):
//   randomize-then-orthogonalize with a random TT Omega of ranks l given by
//   the caller: right partial contractions W_k of x with Omega, then one
//   left-to-right sweep where the sketch Z = X_k^L W_{k+1} is orthonormalized
//   (shifted Cholesky QR then two unshifted passes, so that Q spans range(Z)
//   whatever its conditioning) and core_{k+1} <- (Q^T X_k^L) core_{k+1}.
//   Ranks become at most l; an optional TT-round at delta follows.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "api_common.h"

namespace ttgb {

namespace {

template <class T>
struct Work {
    tt_ctx* c;
    char* base = nullptr;
    size_t bytes = 0, used = 0;
    Work(tt_ctx* ctx, size_t b) : c(ctx), bytes(b) { base = (char*)ctx->alloc(b); }
    ~Work() { c->release(base, bytes); }
    template <class U>
    U* take(size_t elems) {
        const size_t b = (elems * sizeof(U) + 255) & ~size_t(255);
        if (used + b > bytes) throw_status(TT_ERR_ARG, "internal: workspace exhausted");
        U* p = (U*)(base + used);
        used += b;
        return p;
    }
};

inline size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

template <class T>
constexpr double unit_roundoff() {
    return sizeof(T) == 8 ? 1.1102230246251565e-16 : 5.960464477539063e-08;
}

// minimal rank with discarded root-sum-square <= eps, capped at max_rank
// (> 0); *tail2 receives the discarded sum of squares
int trunc_rank_host(const std::vector<double>& s, double eps, int max_rank, double* tail2) {
    const int p = (int)s.size();
    std::vector<double> tail(p + 1, 0.0);
    for (int i = p - 1; i >= 0; --i) tail[i] = tail[i + 1] + s[i] * s[i];
    int rr = std::max(1, p);
    for (int t = 1; t <= p; ++t)
        if (tail[t] <= eps * eps) {
            rr = t;
            break;
        }
    if (max_rank > 0 && rr > max_rank) rr = max_rank;
    rr = std::min(rr, std::max(1, p));
    *tail2 = p > 0 ? tail[rr] : 0.0;
    return rr;
}

// x *= 1 / sqrt(*ss) when *ss > 0 (a device sum of squares): rescales a
// sketch contraction without a host round trip
template <class T>
__global__ void scale_rsqrt_kernel(T* __restrict__ x, long n, const double* __restrict__ ss) {
    const double v = *ss;
    if (!(v > 0.0) || !isfinite(v)) return;
    const double f = 1.0 / sqrt(v);
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        x[i] = (T)((double)x[i] * f);
}

template <class T>
void read_status(tt_ctx* c, const CholStatus* st, int n) {
    std::vector<CholStatus> h(n);
    TT_CUDA(cudaMemcpyAsync(h.data(), st, n * sizeof(CholStatus), cudaMemcpyDeviceToHost, c->stream));
    c->sync();
    for (auto& s : h)
        if (s.nonfinite) throw_status(TT_ERR_NONFINITE, "NaN or Inf in a Gram matrix");
}

// ------------------------------------------------------------- Gram-SVD
template <class T>
tt_tensor* gram_svd_t(tt_ctx* c, const tt_tensor* x, double delta, int max_rank, double* err_est) {
    const int d = x->d;
    if (d == 1) {
        if (err_est) *err_est = 0.0;
        return copy_tensor(c, x);
    }
    std::vector<int> n(x->n), r(x->r);
    int rmax = 1;
    size_t cap = 1;
    for (int k = 0; k <= d; ++k) rmax = std::max(rmax, r[k]);
    for (int k = 0; k < d; ++k) cap = std::max(cap, x->core_elems(k));
    const size_t rr = (size_t)rmax * rmax;
    const size_t bytes = (d + 1) * al256(cap * sizeof(T)) + (d + 10) * al256(rr * sizeof(T)) +
                         al256(2 * rr * sizeof(double)) + al256(rmax * sizeof(double)) +
                         al256((2 * d + 2) * sizeof(CholStatus)) + 4096;
    Work<T> w(c, bytes);
    std::vector<T*> core(d), GR(d + 1, nullptr);
    for (int k = 0; k < d; ++k) {
        core[k] = w.template take<T>(x->core_elems(k) > 0 ? cap : 1);
        TT_CUDA(cudaMemcpyAsync(core[k], x->cores[k], sizeof(T) * x->core_elems(k), cudaMemcpyDeviceToDevice,
                                c->stream));
    }
    T* spare = w.template take<T>(cap);
    for (int k = 1; k < d; ++k) GR[k] = w.template take<T>(rr);
    T* LL = w.template take<T>(rr);
    T* TL = w.template take<T>(rr);
    T* LR = w.template take<T>(rr);
    T* TR = w.template take<T>(rr);
    T* M = w.template take<T>(rr);
    T* U = w.template take<T>(rr);
    T* SVt = w.template take<T>(rr);
    T* P = w.template take<T>(rr);
    T* G = w.template take<T>(rr);
    double* jwork = w.template take<double>(2 * rr);
    double* sig = w.template take<double>(rmax);
    CholStatus* st = w.template take<CholStatus>(2 * d + 2);
    const double u = unit_roundoff<T>();

    // right Grams: GR[k] (r_k x r_k) of the right part starting at core k
    {
        const int a = r[d - 1];
        const long K = (long)n[d - 1] * r[d];
        gemm<T>(*c, false, true, a, a, (int)K, T(1), core[d - 1], K, core[d - 1], K, T(0), GR[d - 1], a);
        for (int k = d - 2; k >= 1; --k) {
            const int ak = r[k], bk = r[k + 1];
            const long NK = (long)n[k] * bk;
            // T1 = X_k^L (ak n x bk) GR[k+1] (bk x bk), kept in `spare`
            gemm<T>(*c, false, false, ak * n[k], bk, bk, T(1), core[k], bk, GR[k + 1], bk, T(0), spare, bk);
            // GR[k] = T1^R (ak x n bk) X_k^R^T
            gemm<T>(*c, false, true, ak, ak, (int)NK, T(1), spare, NK, core[k], NK, T(0), GR[k], ak);
        }
    }
    double eps = -1.0, err2 = 0.0, nrm = 0.0;
    int nst = 0;
    for (int k = 0; k + 1 < d; ++k) {
        const int a = r[k], b = r[k + 1];
        const int m = a * n[k];
        const long NR = (long)n[k + 1] * r[k + 2];
        // G_L = X_k^L^T X_k^L (cores left of k are orthonormal), lower triangle
        gram<T, T>(*c, false, b, m, core[k], b, G);
        const double drop = 16.0 * b * u;
        chol_inv<T, T>(*c, b, G, LL, TL, 0.0, drop, st + nst++);
        chol_inv<T, T>(*c, b, GR[k + 1], LR, TR, 0.0, drop, st + nst++);
        // M = A^T B = L_L^T L_R
        gemm<T>(*c, true, false, b, b, b, T(1), LL, b, LR, b, T(0), M, b, 1, 0, 0, 0, TRI_A_UPPER | TRI_B_LOWER);
        const double tol = sizeof(T) == 8 ? std::max(1e-15, b * u) : 64.0 * u;
        const double fl = sizeof(T) == 8 ? 4.0 * sqrt((double)b) * u : u;
        jacobi_svd<T>(*c, b, b, M, U, SVt, sig, (T*)jwork, tol, fl);
        std::vector<double> hs(b);
        TT_CUDA(cudaMemcpyAsync(hs.data(), sig, b * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        c->sync();
        if (eps < 0.0) {
            double s2 = 0.0;
            for (double v : hs) s2 += v * v;
            nrm = sqrt(s2);
            if (!isfinite(nrm)) throw_status(TT_ERR_NONFINITE, "NaN or Inf in the tensor");
            eps = delta * nrm / sqrt((double)(d - 1));
        }
        double t2 = 0.0;
        const int rp = trunc_rank_host(hs, eps, max_rank, &t2);
        err2 += t2;
        // core_k <- X_k^L (m x b) (T_L^T U_r) (b x rp)
        gemm<T>(*c, true, false, b, rp, b, T(1), TL, b, U, b, T(0), P, rp);
        gemm<T>(*c, false, false, m, rp, b, T(1), core[k], b, P, rp, T(0), spare, rp);
        std::swap(core[k], spare);
        // core_{k+1} <- (S_r V_r^T T_R) (rp x b) X_{k+1}^R (b x NR)
        gemm<T>(*c, false, false, rp, b, b, T(1), SVt, b, TR, b, T(0), P, b, 1, 0, 0, 0, TRI_B_LOWER);
        gemm<T>(*c, false, false, rp, (int)NR, b, T(1), P, b, core[k + 1], NR, T(0), spare, NR);
        std::swap(core[k + 1], spare);
        r[k + 1] = rp;
    }
    read_status<T>(c, st, nst);
    tt_tensor* y = new_tensor(c, d, n.data(), r.data());
    for (int k = 0; k < d; ++k)
        TT_CUDA(cudaMemcpyAsync(y->cores[k], core[k], sizeof(T) * y->core_elems(k), cudaMemcpyDeviceToDevice,
                                c->stream));
    if (err_est) *err_est = nrm > 0 ? sqrt(err2) / nrm : 0.0;
    c->stats.roundings++;
    return y;
}

// ------------------------------------------------------------- randomized
// Z (rows x l, row-major) is overwritten by an orthonormal basis of its
// column space: a shifted Cholesky QR pass (G + s I, s = 8 sqrt(l) u
// trace G), then two unshifted passes that drop numerically zero pivots
// (their columns become zero).  Each pass: G = Z^T Z, G = L L^T, Z <- Z T^T.
template <class T>
void orthonormalize_cols(tt_ctx* c, int rows, int l, T*& Z, T*& spare, T* G, T* L, T* Tinv, CholStatus* st) {
    const double u = unit_roundoff<T>();
    const double sq = sqrt((double)l);
    for (int pass = 0; pass < 3; ++pass) {
        gram<T, T>(*c, false, l, rows, Z, l, G);
        chol_inv<T, T>(*c, l, G, L, Tinv, pass == 0 ? 8.0 * sq * u : 0.0, pass == 0 ? 0.0 : 8.0 * sq * u, st + pass);
        gemm<T>(*c, false, true, rows, l, l, T(1), Z, l, Tinv, l, T(0), spare, l, 1, 0, 0, 0, TRI_B_UPPER);
        std::swap(Z, spare);
    }
}

template <class T>
tt_tensor* randomized_t(tt_ctx* c, const tt_tensor* x, const tt_tensor* om, double* err_est) {
    const int d = x->d;
    if (d == 1) {
        if (err_est) *err_est = 0.0;
        return copy_tensor(c, x);
    }
    std::vector<int> n(x->n), r(x->r), l(om->r);
    size_t cap = 1, wmax = 1, zmax = 1;
    int lmax = 1;
    for (int k = 0; k < d; ++k) cap = std::max(cap, x->core_elems(k));
    for (int k = 0; k <= d; ++k) {
        lmax = std::max(lmax, l[k]);
        wmax = std::max(wmax, (size_t)r[k] * l[k]);
    }
    // cores after the sweep: core k is min(r_k, l_k)-ish x n x l_{k+1}
    // (rows of Z), core k+1 l_{k+1} x n x r_{k+2}; sizes bounded by
    // max(r, l) products
    for (int k = 0; k < d; ++k) {
        const size_t lo = (size_t)std::max(r[k], l[k]), hi = (size_t)std::max(r[k + 1], l[k + 1]);
        zmax = std::max(zmax, lo * n[k] * hi);
        zmax = std::max(zmax, (size_t)r[k] * n[k] * std::max((size_t)r[k + 1], (size_t)l[k + 1]));
    }
    cap = std::max(cap, zmax);
    const size_t ll = (size_t)lmax * lmax;
    const size_t bytes = (d + 3) * al256(cap * sizeof(T)) + (d + 1) * al256(wmax * sizeof(T)) +
                         3 * al256(ll * sizeof(T)) + al256((3 * d + 3) * sizeof(CholStatus)) +
                         al256((d + 1) * sizeof(double)) + 4096;
    Work<T> w(c, bytes);
    std::vector<T*> core(d), W(d + 1, nullptr);
    for (int k = 0; k < d; ++k) {
        core[k] = w.template take<T>(cap);
        TT_CUDA(cudaMemcpyAsync(core[k], x->cores[k], sizeof(T) * x->core_elems(k), cudaMemcpyDeviceToDevice,
                                c->stream));
    }
    T* spare = w.template take<T>(cap);
    T* Z = w.template take<T>(cap);
    for (int k = 1; k < d; ++k) W[k] = w.template take<T>(wmax);
    T* G = w.template take<T>(ll);
    T* L = w.template take<T>(ll);
    T* Tinv = w.template take<T>(ll);
    CholStatus* st = w.template take<CholStatus>(3 * d + 3);
    double* wss = w.template take<double>(d + 1);
    const T* const* oc = (const T* const*)om->cores.data();
    // each W[k] is scaled to unit Frobenius norm: the column space of the
    // sketch Z = X^L W does not depend on W's scale, and unscaled products of
    // d Gaussian sketch cores overflow FP32
    auto normalize = [&](int k) {
        const long ne = (long)r[k] * l[k];
        sumsq<T>(*c, ne, W[k], wss + k);
        const long want = (ne + 255) / 256;
        scale_rsqrt_kernel<T><<<(unsigned)std::max(1L, std::min(want, (long)std::max(1, c->sm_count) * 4)), 256, 0,
                                c->stream>>>(W[k], ne, wss + k);
        TT_LAUNCHED(*c);
    };

    // W[k] (r_k x l_k) = sum_i X_k(i) W[k+1] Omega_k(i)^T, W[d] = 1
    {
        const int a = r[d - 1], b = l[d - 1];
        const long K = (long)n[d - 1];  // r_d = l_d = 1
        gemm<T>(*c, false, true, a, b, (int)K, T(1), core[d - 1], K, oc[d - 1], K, T(0), W[d - 1], b);
        normalize(d - 1);
        for (int k = d - 2; k >= 1; --k) {
            // V = X_k^L (r_k n x r_{k+1}) W[k+1] (r_{k+1} x l_{k+1})
            gemm<T>(*c, false, false, r[k] * n[k], l[k + 1], r[k + 1], T(1), core[k], r[k + 1], W[k + 1], l[k + 1],
                    T(0), spare, l[k + 1]);
            // W[k] = V^R (r_k x n l_{k+1}) Omega_k^R^T (n l_{k+1} x l_k)
            const long NL = (long)n[k] * l[k + 1];
            gemm<T>(*c, false, true, r[k], l[k], (int)NL, T(1), spare, NL, oc[k], NL, T(0), W[k], l[k]);
            normalize(k);
        }
    }
    int nst = 0;
    for (int k = 0; k + 1 < d; ++k) {
        const int a = r[k], b = r[k + 1], lk = l[k + 1];
        const int m = a * n[k];
        const long NR = (long)n[k + 1] * r[k + 2];
        if (lk >= m) {
            // the sketch spans all m rows (generic Omega): Q = I_m, and the
            // core's left unfolding moves into the next core unchanged
            const long NR2 = NR;
            gemm<T>(*c, false, false, m, (int)NR2, b, T(1), core[k], b, core[k + 1], NR2, T(0), Z, NR2);
            std::swap(core[k + 1], Z);
            fill_identity<T>(*c, m, core[k], m);
            r[k + 1] = m;
            continue;
        }
        // Z = X_k^L (m x b) W[k+1] (b x lk)
        gemm<T>(*c, false, false, m, lk, b, T(1), core[k], b, W[k + 1], lk, T(0), Z, lk);
        orthonormalize_cols<T>(c, m, lk, Z, spare, G, L, Tinv, st + nst);
        nst += 3;
        // core_{k+1} <- (Q^T X_k^L) core_{k+1}: first M = Q^T X_k^L (lk x b)
        T* Mbuf = spare;
        gemm<T>(*c, true, false, lk, b, m, T(1), Z, lk, core[k], b, T(0), Mbuf, b);
        // core_k <- Q (m x lk)
        std::swap(core[k], Z);
        // core_{k+1} (b x NR) <- M (lk x b) core_{k+1}, into Z (free now)
        gemm<T>(*c, false, false, lk, (int)NR, b, T(1), Mbuf, b, core[k + 1], NR, T(0), Z, NR);
        std::swap(core[k + 1], Z);
        r[k + 1] = lk;
    }
    read_status<T>(c, st, nst);
    tt_tensor* y = new_tensor(c, d, n.data(), r.data());
    for (int k = 0; k < d; ++k)
        TT_CUDA(cudaMemcpyAsync(y->cores[k], core[k], sizeof(T) * y->core_elems(k), cudaMemcpyDeviceToDevice,
                                c->stream));
    if (err_est) *err_est = -1.0;  // not estimated by the sketch
    return y;
}

}  // namespace

}  // namespace ttgb

using namespace ttgb;

extern "C" {

tt_status tt_round_gram_svd(tt_ctx* ctx, const tt_tensor* x, double delta, int max_rank, tt_tensor** out,
                            double* err_est) {
    TT_API_BEGIN
    if (!ctx || !out) throw_status(TT_ERR_ARG, "NULL argument");
    *out = nullptr;
    check_tensor(ctx, x);
    if (!(delta >= 0.0) || !isfinite(delta)) throw_status(TT_ERR_ARG, "delta must be finite and >= 0");
    if (max_rank < 0) throw_status(TT_ERR_ARG, "max_rank must be >= 0");
    if (ctx->prec == TT_FP64) *out = gram_svd_t<double>(ctx, x, delta, max_rank, err_est);
    else *out = gram_svd_t<float>(ctx, x, delta, max_rank, err_est);
    TT_API_END
}

tt_status tt_round_randomized(tt_ctx* ctx, const tt_tensor* x, const tt_tensor* omega, double delta,
                              tt_tensor** out) {
    TT_API_BEGIN
    if (!ctx || !out) throw_status(TT_ERR_ARG, "NULL argument");
    *out = nullptr;
    check_tensor(ctx, x);
    check_tensor(ctx, omega);
    check_same_modes(x, omega);
    if (!(delta >= 0.0) || !isfinite(delta)) throw_status(TT_ERR_ARG, "delta must be finite and >= 0");
    tt_tensor* y = ctx->prec == TT_FP64 ? randomized_t<double>(ctx, x, omega, nullptr)
                                        : randomized_t<float>(ctx, x, omega, nullptr);
    if (delta > 0.0) {
        TensorGuard g(y);
        y = round_internal(ctx, g.get(), delta, nullptr);
    }
    *out = y;
    TT_API_END
}

}  // extern "C"
