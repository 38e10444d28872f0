// The six TT orthogonalization schemes (Section 3, Algorithms 1-8) as host
// loops over the GPU primitives: TT dot, rank-concatenating axpy, TT-round,
// norm and scaling.  R is assembled on the host in FP64 (column-major, column
// i holds the coefficients of a_i).
#include <cuda_runtime.h>
#include <math.h>

#include <memory>
#include <vector>

#include "api_common.h"

namespace ttgb {

namespace {

struct Driver {
    tt_ctx* c;
    double delta;
    tt_round_policy pol;
    int nrounds = 0;

    tt_tensor* round(const tt_tensor* p, bool fb32_ok = false) {
        nrounds++;
        return round_internal(c, p, delta, nullptr, nullptr, 0, fb32_ok);
    }
    double dot(const tt_tensor* a, const tt_tensor* b) {
        double v = 0.0;
        const tt_tensor* ys[1] = {b};
        dot_many_internal(c, a, 1, ys, &v);
        return v;
    }
    // p + alpha q by concatenation
    tt_tensor* axpy(const tt_tensor* p, double alpha, const tt_tensor* q) {
        double al[2] = {1.0, alpha};
        const tt_tensor* xs[2] = {p, q};
        return tt_add_internal(c, 2, al, xs);
    }
    double norm(const tt_tensor* p) { return norm_internal(c, p); }
};

// running vector: either borrowed (an input) or owned
struct Cur {
    const tt_tensor* p = nullptr;
    TensorGuard own;
    void set_owned(tt_tensor* t) {
        own.reset(t);  // frees the previous owned tensor after t was computed
        p = t;
    }
};

tt_tensor* normalize(Driver& D, const tt_tensor* p, double* nrm_out) {
    const double nrm = D.norm(p);
    if (!(nrm > 0.0)) throw_status(TT_ERR_BREAKDOWN, "zero vector in normalisation");
    *nrm_out = nrm;
    return scale_internal(D.c, p, 1.0 / nrm);
}

// One outer iteration of Algorithms 1-4: orthogonalizes a against the
// orthonormal Q[0..i-1] and normalises it.  col[0..i-1] receives the
// projection coefficients R(j, i) (the two passes summed when twice, as
// R = R^(1) + R^(2) in Algorithms 3 and 4), col[i] the norm R(i, i).
// Rounding follows the policy: TT_ROUND_PAPER rounds once per pass (and the
// first vector, i = 0, is rounded in both policies); TT_ROUND_EVERY_UPDATE
// after every axpy.
// qgram (may be NULL): the Gram matrix <q_j', q_j> of Q (row-major, leading
// dimension ldg).  With it, a modified pass under the paper policy computes
// its coefficients from one batched set of dots: the running vector of
// Algorithms 2 and 4 is p_prev - sum_{j'<j} r_j' q_j', so by linearity
// r_j = <p_prev, q_j> - sum_{j'<j} r_j' <q_j', q_j>, and the i updates are one
// concatenation (the same TT as the successive axpys).
tt_tensor* gs_step(Driver& D, const tt_tensor* a, int i, const tt_tensor* const* Q, double* col, bool modified,
                   bool twice, const double* qgram = nullptr, int ldg = 0) {
    for (int j = 0; j <= i; ++j) col[j] = 0.0;
    Cur prev;
    prev.p = a;
    std::vector<double> rk(i);
    std::vector<double> al(i + 1);
    std::vector<const tt_tensor*> xs(i + 1);
    for (int k = 0; k < (twice ? 2 : 1); ++k) {
        Cur p;
        p.p = prev.p;
        // the pass's sum keeps at least 1e-2 of ||p_prev||^2 (estimated
        // below from the basis Gram when it is known): no cancellation that
        // FP32 fallbacks of the rounding could not resolve
        bool pass_fb32 = false;
        const bool linear_mgs = modified && qgram && D.pol == TT_ROUND_PAPER && i > 0;
        if ((!modified || linear_mgs) && i > 0) {
            // classical: every projection is against the same vector, so the
            // i dots are one batched call; with one rounding per pass the
            // i axpys are one concatenation [p, q_0, ..., q_{i-1}] with
            // coefficients (1, -r_0, ..., -r_{i-1}), the same TT the
            // successive axpys build
            dot_many_internal(D.c, prev.p, i, Q, rk.data(), true);
            const std::vector<double> cdots(rk);  // <p_prev, q_j>
            if (linear_mgs)
                for (int j = 0; j < i; ++j)
                    for (int jp = 0; jp < j; ++jp) rk[j] -= rk[jp] * qgram[(size_t)jp * ldg + j];
            if (qgram && D.c->prec != TT_FP64) {
                // with the basis Gram at hand (resident bases): the sum
                // p_prev - sum_j r_j q_j keeps ||p||^2 = ||p_prev||^2 - 2 r^T c
                // + r^T G r of ||p_prev||^2 (c the dots); when that share is
                // not small, the rounding's fallbacks may stay in FP32
                const double np = D.norm(prev.p);
                const double n2 = np * np;
                double rc = 0.0, rgr = 0.0;
                for (int j = 0; j < i; ++j) {
                    rc += rk[j] * cdots[j];
                    for (int jp = 0; jp < i; ++jp) rgr += rk[j] * qgram[(size_t)j * ldg + jp] * rk[jp];
                }
                const double left = n2 - 2.0 * rc + rgr;
                pass_fb32 = n2 > 0.0 && left >= 1e-2 * n2;
            }
            if (D.pol == TT_ROUND_PAPER) {
                al[0] = 1.0;
                xs[0] = prev.p;
                for (int j = 0; j < i; ++j) {
                    col[j] += rk[j];
                    al[j + 1] = -rk[j];
                    xs[j + 1] = Q[j];
                }
                p.set_owned(tt_add_internal(D.c, i + 1, al.data(), xs.data()));
            } else {
                for (int j = 0; j < i; ++j) {
                    col[j] += rk[j];
                    p.set_owned(D.axpy(p.p, -rk[j], Q[j]));
                    p.set_owned(D.round(p.p));
                }
            }
        } else {
            for (int j = 0; j < i; ++j) {
                const double rji = D.dot(p.p, Q[j]);
                col[j] += rji;
                p.set_owned(D.axpy(p.p, -rji, Q[j]));
                if (D.pol == TT_ROUND_EVERY_UPDATE) p.set_owned(D.round(p.p));
            }
        }
        if (D.pol == TT_ROUND_PAPER || i == 0) p.set_owned(D.round(p.p, pass_fb32));
        // prev <- p (move ownership)
        if (p.own.get()) {
            prev.own = std::move(p.own);
            prev.p = prev.own.get();
        } else {
            prev.p = p.p;
        }
    }
    double nrm;
    tt_tensor* q = normalize(D, prev.p, &nrm);
    col[i] = nrm;
    return q;
}

// Algorithms 1-4 (modified: MGS variants; twice: the reorthogonalized ones)
void gs(Driver& D, int m, const tt_tensor* const* A, std::vector<TensorGuard>& Q, double* R, bool modified,
        bool twice) {
    std::vector<const tt_tensor*> qp(m, nullptr);
    for (int i = 0; i < m; ++i) {
        Q[i].reset(gs_step(D, A[i], i, qp.data(), R + (size_t)i * m, modified, twice));
        qp[i] = Q[i].get();
    }
}

// Algorithm 5: Gram matrix from TT dots, Cholesky and explicit inverse on the
// GPU (FP64), q_i = sum_{k<=i} R^{-1}(k,i) a_k, one rounding per i.
void gram_scheme(Driver& D, int m, const tt_tensor* const* A, std::vector<TensorGuard>& Q, double* R) {
    std::vector<double> G((size_t)m * m);
    for (int i = 0; i < m; ++i) {
        std::vector<double> v(i + 1);
        dot_many_internal(D.c, A[i], i + 1, A, v.data());
        for (int j = 0; j <= i; ++j) G[(size_t)i * m + j] = G[(size_t)j * m + i] = v[j];
    }
    tt_ctx* c = D.c;
    const size_t mm = (size_t)m * m;
    const size_t bytes = 3 * mm * sizeof(double) + sizeof(CholStatus) + 256;
    char* ws = (char*)c->alloc(bytes);
    struct Rel {
        tt_ctx* c; void* p; size_t b;
        ~Rel() { c->release(p, b); }
    } rel{c, ws, bytes};
    double* dG = (double*)ws;
    double* dL = dG + mm;
    double* dT = dL + mm;
    CholStatus* st = (CholStatus*)(dT + mm);
    TT_CUDA(cudaMemcpyAsync(dG, G.data(), mm * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    chol_inv<double, double>(*c, m, dG, dL, dT, 0.0, 0.0, st);
    std::vector<double> L(mm), T(mm);
    CholStatus hs;
    TT_CUDA(cudaMemcpyAsync(L.data(), dL, mm * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    TT_CUDA(cudaMemcpyAsync(T.data(), dT, mm * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    TT_CUDA(cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, c->stream));
    c->sync();
    if (hs.nonfinite) throw_status(TT_ERR_NONFINITE, "NaN or Inf in the Gram matrix");
    if (hs.ndrop) throw_status(TT_ERR_NOT_SPD, "Cholesky of the Gram matrix failed");
    // R = L^T (column-major: R(j,i) = L(i,j)); R^{-1} = (L^{-1})^T: Rinv(k,i) = T(i,k)
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) R[j + (size_t)i * m] = L[(size_t)i * m + j];
    for (int i = 0; i < m; ++i) {
        Cur p;
        p.set_owned(scale_internal(c, A[0], T[(size_t)i * m + 0]));
        for (int j = 1; j <= i; ++j) {
            p.set_owned(D.axpy(p.p, T[(size_t)i * m + j], A[j]));
            if (D.pol == TT_ROUND_EVERY_UPDATE) p.set_owned(D.round(p.p));
        }
        if (D.pol == TT_ROUND_PAPER || i == 0) p.set_owned(D.round(p.p));
        Q[i].reset(p.own.release());
    }
}

// canonical e_j (Section 3.3): rank 1, a single 1 at phi(j), i_1 fastest
tt_tensor* canonical(tt_ctx* c, const std::vector<int>& n, long j) {
    const int d = (int)n.size();
    std::vector<int> r(d + 1, 1);
    tt_tensor* e = new_tensor(c, d, n.data(), r.data());
    long t = j;
    for (int k = 0; k < d; ++k) {
        const int ik = (int)(t % n[k]);
        t /= n[k];
        const size_t es = dtype_size(e->dtype);
        TT_CUDA(cudaMemsetAsync(e->cores[k], 0, es * n[k], c->stream));
        if (e->dtype == TT_DTYPE_F64) {
            static const double one = 1.0;
            TT_CUDA(cudaMemcpyAsync((double*)e->cores[k] + ik, &one, 8, cudaMemcpyHostToDevice, c->stream));
        } else {
            static const float one = 1.0f;
            TT_CUDA(cudaMemcpyAsync((float*)e->cores[k] + ik, &one, 4, cudaMemcpyHostToDevice, c->stream));
        }
    }
    e->norm_hint = 1.0;
    return e;
}

tt_tensor* apply_h(Driver& D, const tt_tensor* a, const tt_tensor* u) {
    const double s = D.dot(a, u);
    return D.axpy(a, -2.0 * s, u);
}

// Algorithm 6
tt_tensor* tth_vec(Driver& D, const tt_tensor* a, const std::vector<TensorGuard>& E, int i, double* r) {
    double s = 0.0;
    Cur w;
    w.p = a;
    for (int j = 0; j < i - 1; ++j) {
        r[j] = D.dot(a, E[j].get());
        s += r[j] * r[j];
        w.set_owned(D.axpy(w.p, -r[j], E[j].get()));
    }
    w.set_owned(D.round(w.p));
    const double na = D.norm(a);
    double t = na * na - s;
    if (t < 0.0) t = 0.0;
    const double fi = D.dot(a, E[i - 1].get());
    const double sg = fi >= 0.0 ? 1.0 : -1.0;
    r[i - 1] = (D.c->sign_rule == TT_SIGN_STABLE ? -sg : sg) * sqrt(t);
    w.set_owned(D.axpy(w.p, -r[i - 1], E[i - 1].get()));
    w.set_owned(D.round(w.p));
    double nw;
    return normalize(D, w.p, &nw);
}

// Algorithm 8, first loop: the Householder TT-vectors u_1..u_m and R (the
// reflections of the a_j); E receives the canonical e_1..e_m
void householder_vectors(Driver& D, int m, const tt_tensor* const* A, std::vector<TensorGuard>& E,
                         std::vector<TensorGuard>& U, double* R) {
    const std::vector<int>& n = A[0]->n;
    double prodn = 1.0;
    for (int v : n) prodn *= v;
    if (prodn < m) throw_status(TT_ERR_ARG, "prod(n) must be >= m for the canonical basis");
    E.resize(m);
    for (int j = 0; j < m; ++j) E[j].reset(canonical(D.c, n, j));
    std::vector<Cur> a(m);
    for (int j = 0; j < m; ++j) a[j].p = A[j];
    U.resize(m);
    Cur w;
    w.set_owned(D.round(A[0]));
    std::vector<double> r(m);
    for (int i = 0; i < m; ++i) {
        U[i].reset(tth_vec(D, w.p, E, i + 1, r.data()));
        for (int j = 0; j <= i; ++j) R[j + (size_t)i * m] = r[j];
        for (int j = i; j < m; ++j) {
            a[j].set_owned(apply_h(D, a[j].p, U[i].get()));
            if (D.pol == TT_ROUND_EVERY_UPDATE && j > i) a[j].set_owned(D.round(a[j].p));
        }
        if (i < m - 1) w.set_owned(D.round(a[i + 1].p));
    }
}

// Algorithm 8: the vectors and R, then q_i = H_1 ... H_i e_i, rounded
void householder(Driver& D, int m, const tt_tensor* const* A, std::vector<TensorGuard>& Q, double* R) {
    std::vector<TensorGuard> E, U;
    householder_vectors(D, m, A, E, U, R);
    for (int i = 0; i < m; ++i) {
        Cur q;
        q.p = E[i].get();
        for (int j = i; j >= 0; --j) q.set_owned(apply_h(D, q.p, U[j].get()));
        Q[i].reset(D.round(q.p));
    }
}

}  // namespace

tt_tensor* orth_step_internal(tt_ctx* ctx, tt_scheme scheme, double delta, tt_round_policy policy,
                              const tt_tensor* a, int k, const tt_tensor* const* Q, double* col, int* nrounds,
                              const double* qgram, int ldg) {
    if (scheme != TT_CGS && scheme != TT_MGS && scheme != TT_CGS2 && scheme != TT_MGS2)
        throw_status(TT_ERR_ARG, "an orthogonalization step takes TT_CGS, TT_MGS, TT_CGS2 or TT_MGS2");
    Driver D{ctx, delta, policy, 0};
    tt_tensor* q = gs_step(D, a, k, Q, col, scheme == TT_MGS || scheme == TT_MGS2,
                           scheme == TT_CGS2 || scheme == TT_MGS2, qgram, ldg);
    if (nrounds) *nrounds = D.nrounds;
    return q;
}

}  // namespace ttgb

using namespace ttgb;

extern "C" tt_status tt_canonical(tt_ctx* ctx, int d, const int* n, long j, tt_tensor** out) {
    TT_API_BEGIN
    if (!ctx || !out || d < 1 || !n) throw_status(TT_ERR_ARG, "bad arguments");
    *out = nullptr;
    double prodn = 1.0;
    for (int k = 0; k < d; ++k) {
        if (n[k] < 1) throw_status(TT_ERR_ARG, "mode size < 1");
        prodn *= n[k];
    }
    if (j < 0 || (double)j >= prodn) throw_status(TT_ERR_ARG, "index beyond prod(n)");
    *out = canonical(ctx, std::vector<int>(n, n + d), j);
    TT_API_END
}

extern "C" tt_status tt_householder_vectors(tt_ctx* ctx, double delta, tt_round_policy policy, int m,
                                            const tt_tensor* const* A, tt_tensor** U, double* R, int* n_rounds) {
    TT_API_BEGIN
    if (!ctx || !A || !U || !R || m < 1) throw_status(TT_ERR_ARG, "bad arguments");
    for (int i = 0; i < m; ++i) U[i] = nullptr;
    if (!(delta >= 0.0) || !isfinite(delta)) throw_status(TT_ERR_ARG, "delta must be finite and >= 0");
    if (policy != TT_ROUND_PAPER && policy != TT_ROUND_EVERY_UPDATE) throw_status(TT_ERR_ARG, "bad policy");
    for (int i = 0; i < m; ++i) {
        check_tensor(ctx, A[i]);
        check_same_modes(A[0], A[i]);
    }
    Driver D{ctx, delta, policy, 0};
    std::vector<TensorGuard> E, Ug;
    std::vector<double> Rh((size_t)m * m, 0.0);
    householder_vectors(D, m, A, E, Ug, Rh.data());
    for (size_t e = 0; e < Rh.size(); ++e) R[e] = Rh[e];
    for (int i = 0; i < m; ++i) U[i] = Ug[i].release();
    if (n_rounds) *n_rounds = D.nrounds;
    TT_API_END
}

extern "C" tt_status tt_householder_apply(tt_ctx* ctx, int k, const tt_tensor* const* U, const tt_tensor* x,
                                          int transpose, double delta, tt_tensor** out) {
    TT_API_BEGIN
    if (!ctx || !out || k < 0 || (k > 0 && !U)) throw_status(TT_ERR_ARG, "bad arguments");
    *out = nullptr;
    check_tensor(ctx, x);
    for (int j = 0; j < k; ++j) {
        check_tensor(ctx, U[j]);
        check_same_modes(x, U[j]);
    }
    if (isnan(delta) || isinf(delta)) throw_status(TT_ERR_ARG, "delta must be finite");
    Driver D{ctx, delta, TT_ROUND_PAPER, 0};
    Cur y;
    y.p = x;
    for (int t = 0; t < k; ++t) {
        const int j = transpose ? t : k - 1 - t;
        y.set_owned(apply_h(D, y.p, U[j]));
        if (delta >= 0.0) y.set_owned(D.round(y.p));
    }
    *out = y.own.get() ? y.own.release() : copy_tensor(ctx, x);
    TT_API_END
}

extern "C" tt_status tt_orthogonalize(tt_ctx* ctx, tt_scheme scheme, double delta, tt_round_policy policy, int m,
                                      const tt_tensor* const* A, tt_tensor** Q, double* R, int* n_rounds) {
    TT_API_BEGIN
    if (!ctx || !A || !Q || !R || m < 1) throw_status(TT_ERR_ARG, "bad arguments");
    for (int i = 0; i < m; ++i) Q[i] = nullptr;
    if (!(delta >= 0.0) || !isfinite(delta)) throw_status(TT_ERR_ARG, "delta must be finite and >= 0");
    if (policy != TT_ROUND_PAPER && policy != TT_ROUND_EVERY_UPDATE) throw_status(TT_ERR_ARG, "bad policy");
    for (int i = 0; i < m; ++i) {
        check_tensor(ctx, A[i]);
        check_same_modes(A[0], A[i]);
    }
    Driver D{ctx, delta, policy, 0};
    std::vector<TensorGuard> Qg(m);
    std::vector<double> Rh((size_t)m * m, 0.0);
    switch (scheme) {
        case TT_CGS: gs(D, m, A, Qg, Rh.data(), false, false); break;
        case TT_MGS: gs(D, m, A, Qg, Rh.data(), true, false); break;
        case TT_CGS2: gs(D, m, A, Qg, Rh.data(), false, true); break;
        case TT_MGS2: gs(D, m, A, Qg, Rh.data(), true, true); break;
        case TT_GRAM: gram_scheme(D, m, A, Qg, Rh.data()); break;
        case TT_HOUSEHOLDER: householder(D, m, A, Qg, Rh.data()); break;
        default: throw_status(TT_ERR_ARG, "bad scheme");
    }
    for (size_t e = 0; e < Rh.size(); ++e) R[e] = Rh[e];
    for (int i = 0; i < m; ++i) Q[i] = Qg[i].release();
    if (n_rounds) *n_rounds = D.nrounds;
    TT_API_END
}
