// TT-rounding (Section 2: TT-round(x, delta), ||x - x~|| <= delta ||x||) and
// the TT norm, on the GPU.
//
// Right-to-left sweep: each right unfolding X (r_{k-1} x n_k r_k) is
// factored X = L Q with Q row-orthonormal by Cholesky QR passes: Gram
// G = X X^T, G = L L^T, Q = L^{-1} X.  When the first Cholesky is healthy,
// the Gram of its Q is I + E with E of the order of the first pass's
// rounding.  The second pass is then either skipped (the first pass's
// Q is kept, orthonormal to ||E||_F, while the summed ||E||_F of the kept
// passes stays within a budget that bounds their effect on the rounding by
// a small multiple of the storage precision), or Q <- (I + E)^(-1/2) Q with
// the factor (I + E)^(1/2) from the cubic Taylor series (valid while its
// remainder is below the storage precision; checked once per rounding), or
// a second Cholesky pass when the series is off.  An unhealthy first pass
// gives three passes of which the first is shifted (G + s I), with
// numerically dependent rows dropped.  L is absorbed into core k-1; the
// series transform of the right-to-left sweep is folded into the
// left-to-right sweep's absorb.  ||x|| = ||core_1||_F.
// Left-to-right sweep: each left unfolding X (r_{k-1} n_k x r_k) is factored
// X = Q R the same way (on columns); the bond keeps its rank when a
// certified lower bound of sigma_min(R) exceeds 2 eps, else R is decomposed
// by one-sided Jacobi SVD and truncated to the minimal rank whose discarded
// singular values have root-sum-square <= eps = delta ||x|| / sqrt(d - 1).
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <deque>
#include <memory>
#include <vector>

#include "api_common.h"

namespace ttgb {

namespace {

template <class T>
struct Rounder {
    tt_ctx* c;
    int d;
    std::vector<int> n, r;
    bool tc = false;         // tensor-core TF32 Gram on the fast path
    double ug_fast, ug_fb;   // unit round-off of the fast / fallback Gram
    int rmax = 1;
    size_t cap = 1;          // elements per core buffer
    char* ws = nullptr;
    size_t ws_bytes = 0;
    std::vector<T*> core;
    T* spare = nullptr;
    T *G, *Lf[3], *Ti[3], *Lp, *Tmp, *Ub, *SVt, *Mp;
    // Deferred second-pass transforms of the right-to-left sweep: core k
    // holds Q1 and the orthonormal core is Pend[k] * Q1 (Pend[k] is
    // r_{k-1} x r_{k-1}); the left-to-right sweep folds Pend[k] into the
    // matrix it absorbs into core k, an r x r product instead of a second
    // apply over the whole core
    T* Pend;
    std::vector<char> pend;
    double* jwork;
    double* sig;
    double* dsc;             // device scalars
    CholStatus* st;          // per-Cholesky statuses of this rounding
    int nst = 0, st_cap = 0;
    double err2 = 0.0;       // accumulated discarded tail (squared, absolute)
    bool series = true;      // second Cholesky QR passes by the series
    bool series_used = false;
    bool fb32_ok = false;      // FP32 data: fallbacks may stay in FP32 (see orth)
    double skip_budget = 0.0;  // second passes are skipped (first pass kept
                               // alone) while the sum of their ||E||_F stays
                               // within this budget (0: never, e.g. for norms)
    int max_rank = 0;          // rank cap of the left-to-right truncation (0: none)
    bool capped(int b) const { return max_rank > 0 && b > max_rank; }

    Rounder(tt_ctx* ctx, const tt_tensor* x, bool pipelined = false)
        : c(ctx), d(x->d), n(x->n), r(x->r), pipe(pipelined) {
        const bool is64 = sizeof(T) == 8;
        tc = (ctx->prec == TT_MIXED_TF32) && ctx->use_tc;
        ug_fb = is64 ? 1.1102230246251565e-16 : 5.960464477539063e-08;
        ug_fast = tc ? 9.765625e-04 : ug_fb;  // TF32 keeps 10 explicit mantissa bits
        for (int k = 0; k <= d; ++k) rmax = std::max(rmax, r[k]);
        for (int k = 0; k < d; ++k) cap = std::max(cap, x->core_elems(k));
        const size_t rr = (size_t)rmax * rmax;
        st_cap = 16 * d + 16;
        auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
        const size_t core_b = al(cap * sizeof(T));
        const size_t small_b = al(rr * sizeof(T));
        ws_bytes = workspace_bytes(d, rmax, cap, sizeof(T), pipe);
        ws = (char*)ctx->alloc(ws_bytes);
        char* p = ws;
        core.resize(d);
        for (int k = 0; k < d; ++k) { core[k] = (T*)p; p += core_b; }
        spare = (T*)p; p += core_b;
        G = (T*)p; p += small_b;
        for (int i = 0; i < 3; ++i) { Lf[i] = (T*)p; p += small_b; }
        for (int i = 0; i < 3; ++i) { Ti[i] = (T*)p; p += small_b; }
        Lp = (T*)p; p += small_b;
        Tmp = (T*)p; p += small_b;
        Ub = (T*)p; p += small_b;
        SVt = (T*)p; p += small_b;
        Mp = (T*)p; p += small_b;
        Pend = (T*)p; p += (size_t)d * small_b;
        pend.assign(d + 1, 0);
        jwork = (double*)p; p += al(2 * rr * sizeof(double));
        sig = (double*)p; p += al(rmax * sizeof(double));
        dsc = (double*)p; p += al(16 * sizeof(double));
        series = ctx->use_series;
        TT_CUDA(cudaMemsetAsync(dsc, 0, 16 * sizeof(double), c->stream));
        st = (CholStatus*)p;
        p += al((size_t)st_cap * sizeof(CholStatus));
        if (pipe) {
            for (int i = 0; i < kPool; ++i) { freeb.push_back((T*)p); p += core_b; }
            for (int i = 0; i < kDepth; ++i) {
                Lq[i] = (T*)p; p += small_b;
                Tq[i] = (T*)p; p += small_b;
                Gq[i] = (T*)p; p += small_b;
                Eq[i] = (T*)p; p += small_b;
                Rq[i] = (T*)p; p += small_b;
            }
            dq = (double*)p;
            hw = static_cast<HostSlot*>(c->pinned_words());
        }
        // the right-to-left sweep starts at the last cores: with the
        // pipeline, cores d-3 .. 0 are copied on the second stream (last
        // first) while the first bonds run, each bond waiting for the
        // copies of the cores it touches
        const int side_from = pipe ? d - 3 : -1;
        for (int k = d - 1; k > side_from; --k)
            TT_CUDA(cudaMemcpyAsync(core[k], x->cores[k], sizeof(T) * x->core_elems(k), cudaMemcpyDeviceToDevice,
                                    c->stream));
        if (side_from >= 0) {
            copy_ev.assign(d, nullptr);
            cudaEvent_t start = c->event();
            TT_CUDA(cudaEventRecord(start, c->stream));
            OnSide os(c);
            side_used = true;
            TT_CUDA(cudaStreamWaitEvent(c->stream, start, 0));
            c->ev_pool.push_back(start);
            for (int k = side_from; k >= 0; --k) {
                TT_CUDA(cudaMemcpyAsync(core[k], x->cores[k], sizeof(T) * x->core_elems(k),
                                        cudaMemcpyDeviceToDevice, c->stream));
                copy_ev[k] = c->event();
                TT_CUDA(cudaEventRecord(copy_ev[k], c->stream));
            }
        }
    }

    // the critical stream waits for core k's copy (pipelined construction)
    std::vector<cudaEvent_t> copy_ev;
    void await_core(int k) {
        if (k < 0 || k >= (int)copy_ev.size() || !copy_ev[k]) return;
        TT_CUDA(cudaStreamWaitEvent(c->stream, copy_ev[k], 0));
        c->ev_pool.push_back(copy_ev[k]);
        copy_ev[k] = nullptr;
    }
    ~Rounder() {
        // the second stream's work and the host copies still reading the
        // workspace's cores finish first
        for (int i = 0; i < 3; ++i) {
            if (!(i == 0 ? side_used : i == 1 ? tail_used : crit2_used)) continue;
            cudaStream_t sj = i == 0 ? c->side_stream : i == 1 ? c->tail_stream : c->crit2_stream;
            cudaEvent_t e = nullptr;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) {
                cudaEventRecord(e, sj);
                cudaStreamWaitEvent(c->stream, e, 0);
                cudaEventDestroy(e);
            } else {
                cudaStreamSynchronize(sj);
            }
        }
        if (copied) cudaStreamSynchronize(c->copy_stream);
        if (ev_norm) c->ev_pool.push_back(ev_norm);
        for (cudaEvent_t e : copy_ev)
            if (e) c->ev_pool.push_back(e);
        for (cudaEvent_t e : copy_events) c->ev_pool.push_back(e);
        if (ws) c->release(ws, ws_bytes);
        if (ws64) c->release(ws64, ws64_bytes);
    }

    // Host destinations of the output cores (storage type, null: none):
    // each core is copied as soon as the left-to-right sweep has finished
    // it, on the context's copy stream, overlapping the rest of the sweep.
    void* const* host_out = nullptr;
    bool copied = false;
    std::vector<cudaEvent_t> copy_events;
    // ready: core k is already complete on the device (the host has waited
    // for the event that follows its last write)
    void stream_core(int k, bool ready = false) {
        if (!host_out) return;
        cudaStream_t cs = c->copies();
        if (!ready) {
            cudaEvent_t ev = c->event();
            copy_events.push_back(ev);
            TT_CUDA(cudaEventRecord(ev, c->stream));
            TT_CUDA(cudaStreamWaitEvent(cs, ev, 0));
        }
        const size_t bytes = sizeof(T) * (size_t)r[k] * n[k] * r[k + 1];
        TT_CUDA(cudaMemcpyAsync(host_out[k], core[k], bytes, cudaMemcpyDeviceToHost, cs));
        copied = true;
    }

    // bytes of the workspace carved in the constructor (d + 1 core buffers,
    // 12 + d r x r matrices, Jacobi work, singular values, scalars, statuses)
    // (+ with pipelined sweeps: kPool core buffers, 5 kDepth r x r matrices
    // and 8 kDepth device words)
    static size_t workspace_bytes(int d, int rmax, size_t cap, size_t es, bool pipelined = false) {
        auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
        const size_t rr = (size_t)rmax * rmax;
        const size_t base = (d + 1) * al(cap * es) + (12 + d) * al(rr * es) + al(2 * rr * sizeof(double)) +
                            al(rmax * sizeof(double)) + al(16 * sizeof(double)) +
                            al((16 * d + 16) * sizeof(CholStatus));
        return base + (pipelined ? kPool * al(cap * es) + 5 * kDepth * al(rr * es) + al(8 * kDepth * sizeof(double))
                                 : 0);
    }

    CholStatus* next_st() {
        if (nst >= st_cap) throw_status(TT_ERR_ARG, "internal: status slots exhausted");
        return st + nst++;
    }

    CholStatus read_st(CholStatus* s) {
        CholStatus h;
        TT_CUDA(cudaMemcpyAsync(&h, s, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
        c->sync();
        if (h.nonfinite) throw_status(TT_ERR_NONFINITE, "NaN or Inf in a Gram matrix");
        return h;
    }

    void gram_into(bool rows, bool fast, int a, long K, const T* X, T* dst = nullptr) {
        T* Gd = dst ? dst : G;
        if constexpr (sizeof(T) == 4) {
            if (fast && tc) {
                if (rows && gram_rows_tc_tf32(*c, a, K, (const float*)X, K, (float*)Gd)) return;
                if (!rows && gram_cols_tc_tf32(*c, a, K, (const float*)X, a, (float*)Gd)) return;
            }
        }
        gram<T, T>(*c, rows, a, K, X, rows ? K : a, Gd);
    }

    // C = op(A) op(B): tensor-core split TF32 when the context allows it and
    // the layout is TMA-aligned, else the CUDA-core kernel of the storage type
    void mm(bool tA, bool tB, int M, int N, int K, const T* A, long lda, const T* B, long ldb, T* C, long ldc,
            int tri = 0, bool absorb = false) {
        if constexpr (sizeof(T) == 4) {
            if (tc && (c->use_tc_gemm || (absorb && c->use_tc_absorb)) && !tA &&
                gemm_tc3_tf32(*c, tB, M, N, K, (const float*)A, lda, (const float*)B, ldb, (float*)C, ldc,
                              c->tc_gemm_split))
                return;
        }
        gemm<T>(*c, tA, tB, M, N, K, T(1), A, lda, B, ldb, T(0), C, ldc, 1, 0, 0, 0, tri);
    }

    // a Cholesky QR pass's product X <- L_p^{-1} X (or X L_p^{-T}): FP64 data
    // by substitution with L_p (backward stable whatever kappa(L_p): the
    // explicit inverse's error grows like kappa(L) u, which an
    // ill-conditioned unfolding's content does not survive), FP32 data with
    // the explicit inverse T_p (its kappa stays below 1/sqrt(100 u_32) on the
    // fast path, and the FP32 fallback keeps only healthy pivots)
    void apply_factor(bool rows, int a, long K, T*& X, int p) {
        if constexpr (sizeof(T) == 8) {
            trsm_lower<T>(*c, rows, a, K, Lf[p], X, spare);
            std::swap(X, spare);
        } else {
            apply(rows, a, K, X, Ti[p]);
        }
    }

    // X <- Ti X (rows) or X Ti^T (cols); Ti lower-triangular unless !tri
    void apply(bool rows, int a, long K, T*& X, const T* Tinv, bool tri = true) {
        if (rows) mm(false, false, a, (int)K, a, Tinv, a, X, K, spare, K, tri ? TRI_A_LOWER : 0);
        else mm(false, true, (int)K, a, a, X, a, Tinv, a, spare, a, tri ? TRI_B_UPPER : 0);
        std::swap(X, spare);
    }

    struct Orth {
        int npass;
        int ndrop;
        bool shifted;
        int nchol = 0;        // Cholesky passes (factors Lf/Ti[0..nchol)) of the certificate
        bool series = false;  // the second pass was the series pass (||E||_F^2 in dsc[12])
        bool lower = true;    // Lp lower-triangular
        bool deferred = false;  // X holds Q1; the orthonormal factor is S Q1 (S in the defer slot)
        bool series_pending = false;  // E measured, S / R2 / Lp not formed yet
        double e = 0.0;               // ||E||_F of a series pass
        double lb = -1.0;             // certificate bound formed by orth (lr, series), else < 0
    };

    // The series pass is of order 3: valid while the Taylor remainders of
    // (1 + x)^(-1/2) and (1 + x)^(1/2) after the cubic terms, together at
    // most (35 + 5) / 128 e^4 / (1 - e) for ||E||_F = e, stay below the
    // storage precision's unit round-off (e <= 0.021 FP32, 1.4e-4 FP64).
    bool series_valid(double e) const { return e < 0.25 && 0.3125 * pow(e, 4) / (1.0 - e) <= ug_fb; }

    // X (a x K rows, or K x a cols) is overwritten by its orthonormal factor;
    // Lp receives L with X_old = L Q (rows) or X_old = Q L^T (cols), lower-
    // triangular unless the second pass was the series pass (o.lower).
    // Lf[i], Ti[i] keep the factors of each pass.
    // Completes a series second pass whose E (in Ti[1]) and ||E||_F^2 (in
    // dsc[12]) are in place: S over Ti[1], R2 in Lf[1], X <- S X (rows) or
    // X S (cols) unless deferred, Lp = L1 R2.
    void finish_series(bool rows, int a, long K, T*& X, T* defer, Orth& o) {
        c->stats.series_passes++;
        series_used = true;
        mm(false, false, a, a, a, Ti[1], a, Ti[1], a, Lf[1], a);
        mm(false, false, a, a, a, Lf[1], a, Ti[1], a, Tmp, a);
        poly_pair<T>(*c, a, 3, Ti[1], Lf[1], Tmp, Lf[1], dsc + 12, dsc + 11);
        if (defer) {
            // X keeps Q1; S Q1 is formed by the caller's later products
            // (rows only: S acts on the row index)
            TT_CUDA(cudaMemcpyAsync(defer, Ti[1], sizeof(T) * (size_t)a * a, cudaMemcpyDeviceToDevice, c->stream));
            o.deferred = true;
        } else {
            apply(rows, a, K, X, Ti[1], false);
        }
        mm(false, false, a, a, a, Lf[0], a, Lf[1], a, Lp, a, TRI_A_LOWER);
        o.series_pending = false;
        o.lower = false;
    }

    // The first pass's product and the second pass's Gram (and E, and for
    // the left-to-right sweep the first factor's certificate norms) are
    // launched before the first factorization's health is known: one
    // synchronization reads all of it.  An unhealthy first pass restores
    // the original X (kept in `spare` by the apply) and takes the shifted
    // path.  With the series on, a pass whose ||E||_F fits *budget keeps the
    // first pass alone (right-to-left: no certificate needed; `lr`: the
    // caller decides after the certificate, o.series_pending); otherwise the
    // series pass completes (finish_series).
    Orth orth(bool rows, int a, long K, T*& X, T* defer = nullptr, double* budget = nullptr, bool lr = false) {
        const double sq = sqrt((double)a);
        const double drop_fb = 8.0 * ug_fb * sq;
        const double ratio_fast = tc ? 10.0 * ug_fast : 100.0 * ug_fast;
        Orth o{0, 0, false};
        {
            gram_into(rows, true, a, K, X);
            CholStatus* s0 = next_st();
            // drop only numerically-zero pivots here; health is judged by
            // pivot / own diagonal, which Cholesky QR is invariant to
            // (column or row scaling does not change it)
            chol_inv<T, T>(*c, a, G, Lf[0], Ti[0], 0.0, drop_fb, s0);
            apply_factor(rows, a, K, X, 0);
            // the second pass's Gram: a TF32 Gram of the nearly
            // orthonormal X measures E to about u_tf32 / sqrt(K), so
            // it leaves Q orthonormal to that (not to FP32 level); the
            // factorization X = L Q itself stays exact to FP32 rounding
            // (S and R come from the same E).  On tensor cores for long
            // unfoldings (K >= kTc2MinK: defect <= 8e-6), else FP32.
            gram_into(rows, K >= kTc2MinK, a, K, X);
            if (series) near_identity<T>(*c, a, G, Ti[1], dsc + 12);
            if (lr && series) {
                TT_CUDA(cudaMemsetAsync(dsc, 0, 2 * sizeof(double), c->stream));
                inv_and_identity_defect<T>(*c, a, Lf[0], Ti[0], dsc);
            }
            CholStatus h;
            double hd[13] = {0};
            TT_CUDA(cudaMemcpyAsync(&h, s0, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
            TT_CUDA(cudaMemcpyAsync(hd, dsc, 13 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
            c->sync();
            if (h.nonfinite) throw_status(TT_ERR_NONFINITE, "NaN or Inf in a Gram matrix");
            if (h.ndrop == 0 && h.min_ratio >= ratio_fast) {
                o.npass = 2;
                o.nchol = 1;
                if (series) {
                    // G = I + E with E small: Q <- (I + E)^(-1/2) Q and
                    // R = (I + E)^(1/2) from the cubic series in E (two
                    // a x a products instead of a Cholesky factorization;
                    // the factor is symmetric, not triangular).  The
                    // series' validity is checked at the end of the
                    // rounding (one maximum on the device, read with the
                    // statuses); a rounding where ||E||_F was too large is
                    // redone with Cholesky passes.
                    const double e = sqrt(hd[12]);
                    o.series = true;
                    o.series_pending = true;
                    o.e = e;
                    if (lr) {
                        // sigma_min(Q1) >= sqrt(1 - e), sigma_min of the
                        // completed pass's factor likewise (less the series
                        // remainder and the stored factor's rounding)
                        const double lb1 = std::max(hd[0] > 0.0 ? 1.0 / sqrt(hd[0]) : 0.0, 1.0 - sqrt(hd[1]));
                        o.lb = series_valid(e) ? lb1 * std::max(0.0, sqrt(1.0 - e) - (2.0 + sq) * ug_fb) : 0.0;
                        return o;
                    }
                    if (budget && series_valid(e) && e <= *budget) {
                        // Q1 is orthonormal to e: keep it (X = L1 Q1 to
                        // storage rounding); later truncations see
                        // singular values within 1 +- (sum of skipped e)/2
                        *budget -= e;
                        c->stats.second_pass_skips++;
                        TT_CUDA(cudaMemcpyAsync(Lp, Lf[0], sizeof(T) * (size_t)a * a, cudaMemcpyDeviceToDevice,
                                                c->stream));
                        o.series_pending = false;
                        o.lower = true;
                        return o;
                    }
                    finish_series(rows, a, K, X, defer, o);
                    return o;
                }
                chol_inv<T, T>(*c, a, G, Lf[1], Ti[1], 0.0, drop_fb, next_st());
                apply_factor(rows, a, K, X, 1);
                mm(false, false, a, a, a, Lf[0], a, Lf[1], a, Lp, a, TRI_A_LOWER | TRI_B_LOWER);
                o.nchol = 2;
                return o;
            }
            // the first pass's product is discarded: the original X
            std::swap(X, spare);
        }
        // shifted Cholesky QR, then two passes with dependent rows dropped
        c->stats.fallback_orth++;
        o.shifted = true;
        if constexpr (sizeof(T) == 4) {
            // FP32 data: FP64 unless the caller vouched that the tensor
            // being rounded does not cancel far below the scale of its
            // representation (fb32_ok): then the FP32 passes lose nothing
            // the FP32 storage keeps (an exactly rank-deficient concatenation
            // loses only its dependent rows).  Where the tensor cancels (the
            // sums of a Gram-Schmidt scheme on nearly dependent inputs) or
            // its spectrum is graded, FP32 Cholesky QR resolves the content
            // only to about sqrt(u_32) of the unfolding's norm.
            if (!fb32_ok) {
                fallback_fp64(rows, a, K, X, o);
                return o;
            }
            c->stats.fallback_fp32++;
        }
        gram_into(rows, false, a, K, X);
        chol_inv<T, T>(*c, a, G, Lf[0], Ti[0], 8.0 * ug_fb * sq, 0.0, next_st());
        apply_factor(rows, a, K, X, 0);
        for (int p = 1; p <= 2; ++p) {
            gram_into(rows, false, a, K, X);
            chol_inv<T, T>(*c, a, G, Lf[p], Ti[p], 0.0, drop_fb, next_st());
            apply_factor(rows, a, K, X, p);
        }
        mm(false, false, a, a, a, Lf[0], a, Lf[1], a, Tmp, a, TRI_A_LOWER | TRI_B_LOWER);
        mm(false, false, a, a, a, Tmp, a, Lf[2], a, Lp, a, TRI_A_LOWER | TRI_B_LOWER);
        o.npass = 3;
        o.nchol = 3;
        return o;
    }

    // FP64 work buffers of the fallback orthogonalization of FP32 data,
    // allocated on its first use in a rounding
    char* ws64 = nullptr;
    size_t ws64_bytes = 0;
    double *x64 = nullptr, *s64 = nullptr, *G64 = nullptr, *P64 = nullptr, *L64[3] = {}, *T64[3] = {};
    static size_t fallback64_bytes(int rmax, size_t cap) {
        auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
        return 2 * al(cap * sizeof(double)) + 8 * al((size_t)rmax * rmax * sizeof(double));
    }
    void ensure_ws64() {
        if (ws64) return;
        auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
        const size_t rr = (size_t)rmax * rmax;
        ws64_bytes = fallback64_bytes(rmax, cap);
        ws64 = (char*)c->alloc(ws64_bytes);
        char* p = ws64;
        x64 = (double*)p; p += al(cap * sizeof(double));
        s64 = (double*)p; p += al(cap * sizeof(double));
        G64 = (double*)p; p += al(rr * sizeof(double));
        P64 = (double*)p; p += al(rr * sizeof(double));
        for (int i = 0; i < 3; ++i) { L64[i] = (double*)p; p += al(rr * sizeof(double)); }
        for (int i = 0; i < 3; ++i) { T64[i] = (double*)p; p += al(rr * sizeof(double)); }
    }

    // The fallback for FP32 data in FP64 arithmetic: X widened to FP64,
    // shifted Cholesky QR (s = 8 sqrt(a) u_64 trace G) and two unshifted
    // passes dropping only FP64-level zero pivots, Q narrowed back into X and
    // the factors into Lp (and Lf/Ti for the certificate).  Cholesky QR in
    // FP32 loses the content of an unfolding below about sqrt(u_32) of its
    // norm, which for the cancelling sums of the Gram-Schmidt schemes is a
    // large part of the result; in FP64 the loss is at the FP32 storage
    // rounding itself (X = L Q to u_32 ||X||).
    // have_gram: x64 already holds X widened and G64 its Gram (the
    // classification's), so the first pass starts at its Cholesky
    void fallback_fp64(bool rows, int a, long K, T*& X, Orth& o, bool have_gram = false) {
        ensure_ws64();
        const double u64 = 1.1102230246251565e-16;
        const double sq = sqrt((double)a);
        const long nel = (long)a * K;
        if (!have_gram) convert<T, double>(*c, nel, X, x64);
        double* Xd = x64;
        double* Sd = s64;
        for (int p = 0; p < 3; ++p) {
            if (p > 0 || !have_gram) gram<double, double>(*c, rows, a, K, Xd, rows ? K : a, G64);
            chol_inv<double, double>(*c, a, G64, L64[p], T64[p], p == 0 ? 8.0 * u64 * sq : 0.0,
                                     p == 0 ? 0.0 : 8.0 * u64 * sq, next_st());
            // Q = L^{-1} X by substitution (not the explicit inverse): the
            // fallback's unfoldings are the ill-conditioned ones
            trsm_lower<double>(*c, rows, a, K, L64[p], Xd, Sd);
            std::swap(Xd, Sd);
        }
        convert<double, T>(*c, nel, Xd, X);
        gemm<double>(*c, false, false, a, a, a, 1.0, L64[0], a, L64[1], a, 0.0, P64, a, 1, 0, 0, 0,
                     TRI_A_LOWER | TRI_B_LOWER);
        gemm<double>(*c, false, false, a, a, a, 1.0, P64, a, L64[2], a, 0.0, G64, a, 1, 0, 0, 0,
                     TRI_A_LOWER | TRI_B_LOWER);
        convert<double, T>(*c, (long)a * a, G64, Lp);
        for (int i = 0; i < 3; ++i) {
            convert<double, T>(*c, (long)a * a, L64[i], Lf[i]);
            convert<double, T>(*c, (long)a * a, T64[i], Ti[i]);
        }
        o.npass = 3;
        o.nchol = 3;
    }

    // rigorous lower bound of sigma_min(L_0 ... L_{np-1}) from the factors and
    // their inverses: prod_i max(1/||T_i||_F, 1 - ||L_i - I||_F); 0 on drops;
    // times the bound of a series pass's factor
    // (the series passes' bound is formed by orth itself, with its one read)
    double sigma_lb(int a, const Orth& o) {
        const int np = o.nchol;
        TT_CUDA(cudaMemsetAsync(dsc, 0, 2 * np * sizeof(double), c->stream));
        for (int i = 0; i < np; ++i) inv_and_identity_defect<T>(*c, a, Lf[i], Ti[i], dsc + 2 * i);
        std::vector<double> h(2 * np);
        std::vector<CholStatus> hs(nst);
        TT_CUDA(cudaMemcpyAsync(h.data(), dsc, 2 * np * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        TT_CUDA(cudaMemcpyAsync(hs.data(), st, nst * sizeof(CholStatus), cudaMemcpyDeviceToHost, c->stream));
        c->sync();
        for (int i = nst - np; i < nst; ++i) {
            if (hs[i].nonfinite) throw_status(TT_ERR_NONFINITE, "NaN or Inf in a Gram matrix");
            if (hs[i].ndrop) return 0.0;
        }
        double lb = 1.0;
        for (int i = 0; i < np; ++i) {
            double b1 = h[2 * i] > 0 ? 1.0 / sqrt(h[2 * i]) : 0.0;
            double b2 = 1.0 - sqrt(h[2 * i + 1]);
            lb *= std::max(b1, b2);
        }
        return lb;
    }

    // Jacobi tolerances of the truncation SVD.  FP64 storage: rows
    // orthogonal to the rounding floor of a length-b dot product (b u);
    // rows below 4 sqrt(b) u ||R|| are rounding noise.  FP32 storage: R
    // carries FP32 rounding (u_32 relative), so orthogonality beyond
    // 64 u_32 cannot change the data's singular values, and rows below
    // u_32 ||R|| are noise; the SVD still runs in FP64 and its rotations
    // stay exactly orthogonal.
    static double svd_tol(int b) {
        return sizeof(T) == 8 ? std::max(1e-15, b * 1.1102230246251565e-16) : 64.0 * 5.960464477539063e-08;
    }
    static double svd_floor(int b) {
        return sizeof(T) == 8 ? 4.0 * sqrt((double)b) * 1.1102230246251565e-16 : 5.960464477539063e-08;
    }

    // core_{k+1} <- M core_{k+1} (M: rows x r_{k+1}, ld ldm), with core
    // k+1's deferred transform folded in first (M Pend[k+1], r x r)
    // (out: the product's buffer, which becomes core k+1; else spare)
    void absorb_next(int k, int rows, const T* M, long ldm, int tri, T* out = nullptr) {
        const int b = r[k + 1];
        const long NR = (long)n[k + 1] * r[k + 2];
        if (pend[k + 1]) {
            mm(false, false, rows, b, b, M, ldm, Pend + (size_t)(k + 1) * rmax * rmax, b, Mp, b);
            M = Mp;
            ldm = b;
            tri = 0;
            pend[k + 1] = 0;
        }
        if (out) {
            mm(false, false, rows, (int)NR, b, M, ldm, core[k + 1], NR, out, NR, tri, true);
            core[k + 1] = out;
            return;
        }
        mm(false, false, rows, (int)NR, b, M, ldm, core[k + 1], NR, spare, NR, tri, true);
        std::swap(core[k + 1], spare);
    }

    // Truncation of bond k for FP32 data by the FP32 column Jacobi: R (p x b,
    // row-major, ldr = b) with its columns given as the rows of Wsrc (b x p).
    // The kept left vectors U_r are re-orthonormalized (one Cholesky QR pass)
    // and core_{k+1} <- (U_r^T R) core_{k+1}: an exact orthogonal projection.
    // Its error ||R - U_r U_r^T R||_F is measured (FP64 accumulation) and the
    // rank raised until it is <= eps, so the rounding bound holds whatever
    // the FP32 SVD's accuracy; FP32 rotations only cost optimality of the
    // rank near the threshold.  Used for p >= kSvd32Min, where the FP64
    // Jacobi (FP64 runs at 1/64 of the FP32 rate here) takes milliseconds
    // per bond.  qmul: core_k <- core_k U_r
    // (else core_k <- U_r, when Q = I).  False: not taken (nothing done).
    static constexpr int kSvd32Min = 32;
    static constexpr long kTc2MinK = 4096;
    bool trunc_f32(int m, int p, int b, const T* Wsrc, long ldw, const T* R, double eps, int k, long NR,
                   bool qmul) {
        if constexpr (sizeof(T) != 4) {
            return false;
        } else {
            if (p < kSvd32Min) return false;
            if (!jacobi_cols_f32(*c, b, p, Wsrc, ldw, (float*)jwork, (float*)Ub, sig, 8.0 * sqrt((double)p) * ug_fb,
                                 ug_fb))
                return false;
            std::vector<double> hs(b);
            TT_CUDA(cudaMemcpyAsync(hs.data(), sig, b * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
            c->sync();
            const double err2_before = err2;
            int rp = std::min(trunc_rank(hs, eps), p);
            err2 = err2_before;
            T* Uk = Ub;                 // sorted unit columns, p x b (ld b)
            T* Uo = SVt;                // orthonormal U_r, p x rp (ld rp)
            T* S = Tmp == R ? Lf[1] : Tmp;  // U_r^T R, rp x b (ld b)
            T* E = G;                   // R - U_r S
            // FP32 rounding of S = U_r^T R and of R itself leaves about
            // sqrt(p) u_32 ||R|| in any FP32 truncation: the guard accepts
            // residuals within that of eps (it catches SVD subspace errors,
            // not the storage precision)
            sumsq<T>(*c, (long)p * b, R, dsc + 13);
            double r2 = 0.0;
            TT_CUDA(cudaMemcpyAsync(&r2, dsc + 13, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
            double res2 = 0.0;
            for (int attempt = 0;; ++attempt) {
                gram<T, T>(*c, false, rp, p, Uk, b, G);
                chol_inv<T, T>(*c, rp, G, Lf[2], Ti[2], 0.0, 8.0 * ug_fb * sqrt((double)rp), next_st());
                mm(false, true, p, rp, rp, Uk, b, Ti[2], rp, Uo, rp, TRI_B_UPPER);
                mm(true, false, rp, b, p, Uo, rp, R, b, S, b);
                TT_CUDA(cudaMemcpyAsync(E, R, sizeof(T) * (size_t)p * b, cudaMemcpyDeviceToDevice, c->stream));
                gemm<T>(*c, false, false, p, b, rp, T(-1), Uo, rp, S, b, T(1), E, b);
                sumsq<T>(*c, (long)p * b, E, dsc + 14);
                TT_CUDA(cudaMemcpyAsync(&res2, dsc + 14, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
                c->sync();
                const double noise2 = 16.0 * p * ug_fb * ug_fb * r2;
                if (res2 <= eps * eps + noise2 || rp >= p || attempt >= 6 || (max_rank > 0 && rp >= max_rank)) break;
                rp = std::min(p, rp + std::max(1, rp / 8));
                if (max_rank > 0) rp = std::min(rp, max_rank);
            }
            err2 += res2;
            if (qmul) {
                mm(false, false, m, rp, b, core[k], b, Uo, rp, spare, rp);
                std::swap(core[k], spare);
            } else {
                TT_CUDA(cudaMemcpyAsync(core[k], Uo, sizeof(T) * (size_t)p * rp, cudaMemcpyDeviceToDevice, c->stream));
            }
            absorb_next(k, rp, S, b, 0);
            r[k + 1] = rp;
            return true;
        }
    }

    // truncation rank from sorted singular values (FP64, host): the minimal
    // rank whose discarded tail is within eps, then at most max_rank
    int trunc_rank(const std::vector<double>& s, double eps) {
        const int p = (int)s.size();
        if (p < 1) return 1;
        std::vector<double> tail(p + 1, 0.0);
        for (int i = p - 1; i >= 0; --i) tail[i] = tail[i + 1] + s[i] * s[i];
        const double e2 = eps * eps;
        int rr = p;
        for (int t = 1; t <= p; ++t)
            if (tail[t] <= e2) {
                rr = t;
                break;
            }
        if (max_rank > 0 && rr > max_rank) rr = max_rank;
        err2 += tail[rr];
        return rr;
    }

    // bond k of the right-to-left sweep: core k orthonormalized, its factor
    // absorbed into core k-1
    void rl_bond(int k) {
        await_core(k);
        await_core(k - 1);
        const int a = r[k];
        const long K = (long)n[k] * r[k + 1];
        const int M = r[k - 1] * n[k - 1];
        if (K <= a) {
            // rank cap: X = I_K X, absorb X itself
            mm(false, false, M, (int)K, a, core[k - 1], a, core[k], K, spare, K);
            std::swap(core[k - 1], spare);
            fill_identity<T>(*c, (int)K, core[k], K);
            r[k] = (int)K;
        } else {
            const Orth o = orth(true, a, K, core[k], Pend + (size_t)k * rmax * rmax, &skip_budget);
            pend[k] = o.deferred;
            mm(false, false, M, a, a, core[k - 1], a, Lp, a, spare, a, o.lower ? TRI_B_LOWER : 0, true);
            std::swap(core[k - 1], spare);
        }
    }

    void rl_sweep() {
        if (pipe && series && skip_budget > 0.0) {
            rl_sweep_pipelined();
            return;
        }
        for (int k = d - 1; k >= 1; --k) rl_bond(k);
    }

    // ||core_k||_F^2 into device words and a page-locked word, with an event
    cudaEvent_t ev_norm = nullptr;
    void norm_async(int k) {
        sumsq<T>(*c, (long)r[k] * n[k] * r[k + 1], core[k], dsc + 15);
        TT_CUDA(cudaMemcpyAsync(&hw[kDepth].w[0], dsc + 15, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        ev_norm = c->event();
        TT_CUDA(cudaEventRecord(ev_norm, c->stream));
    }
    double nrm_ = -1.0;
    double norm_value() {
        if (nrm_ >= 0.0) return nrm_;
        TT_CUDA(cudaEventSynchronize(ev_norm));
        c->stats.host_syncs++;
        c->ev_pool.push_back(ev_norm);
        ev_norm = nullptr;
        const double h = hw[kDepth].w[0];
        if (!isfinite(h)) throw_status(TT_ERR_NONFINITE, "NaN or Inf in the tensor");
        nrm_ = sqrt(h);
        return nrm_;
    }

    double core_norm(int k) {
        sumsq<T>(*c, (long)r[k] * n[k] * r[k + 1], core[k], dsc + 15);
        double h;
        TT_CUDA(cudaMemcpyAsync(&h, dsc + 15, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        c->sync();
        if (!isfinite(h)) throw_status(TT_ERR_NONFINITE, "NaN or Inf in the tensor");
        return sqrt(h);
    }

    // bond k of the left-to-right sweep: core k orthonormalized (and
    // truncated unless certified), its factor absorbed into core k+1
    void lr_bond(int k, double eps) {
        const int m = r[k] * n[k];
        const int b = r[k + 1];
        const long NR = (long)n[k + 1] * r[k + 2];
        if (m >= b) {
            Orth o = orth(false, b, m, core[k], nullptr, nullptr, true);
            // a capped bond is truncated whatever its spectrum: no certificate
            const bool cap = capped(b);
            const double lb = cap ? 0.0 : (o.lb >= 0.0 ? o.lb : sigma_lb(b, o));
            if (o.series_pending) {
                if (!cap && lb > 2.0 * eps && lb > 0.0 && o.e <= skip_budget) {
                    // certified, and Q1 is orthonormal to ||E||_F: the
                    // bond keeps its rank with core_k = Q1 and
                    // core_{k+1} <- L1^T core_{k+1} (X = Q1 L1^T exactly);
                    // the second pass would only sharpen the cores'
                    // orthonormality.  The left factor of a later bond
                    // then has singular values within 1 +- (sum of the
                    // skipped ||E||_F) / 2, which scales that bond's
                    // truncation error by at most the same factor
                    skip_budget -= o.e;
                    c->stats.certified_bonds++;
                    c->stats.second_pass_skips++;
                    transpose<T>(*c, b, b, Lf[0], Tmp);
                    absorb_next(k, b, Tmp, b, TRI_A_UPPER);
                    return;
                }
                finish_series(false, b, m, core[k], nullptr, o);
            }
            if (lb > 2.0 * eps && lb > 0.0) {
                c->stats.certified_bonds++;
                // core_{k+1} <- R core_{k+1}, R = Lp^T
                transpose<T>(*c, b, b, Lp, Tmp);
                absorb_next(k, b, Tmp, b, o.lower ? TRI_A_UPPER : 0);
                return;
            }
            // R = Lp^T (b x b), SVD, truncate
            transpose<T>(*c, b, b, Lp, Tmp);
            c->stats.svd_calls++;
            // FP32 data: columns of R = rows of Lp, FP32 column Jacobi
            if (trunc_f32(m, b, b, Lp, b, Tmp, eps, k, NR, true)) return;
            jacobi_svd<T>(*c, b, b, Tmp, Ub, SVt, sig, (T*)jwork, svd_tol(b), svd_floor(b));
            std::vector<double> hs(b);
            TT_CUDA(cudaMemcpyAsync(hs.data(), sig, b * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
            c->sync();
            const int rp = trunc_rank(hs, eps);
            mm(false, false, m, rp, b, core[k], b, Ub, b, spare, rp);
            std::swap(core[k], spare);
            absorb_next(k, rp, SVt, b, 0);
            r[k + 1] = rp;
        } else {
            // m < b: Q = I_m, R = X (m x b); certificate from the Gram of
            // the rows of X (SIMT arithmetic, its error is subtracted)
            const T* X = core[k];
            gram<T, T>(*c, true, m, b, X, b, G);
            CholStatus* s = next_st();
            chol_inv<T, T>(*c, m, G, Lf[0], Ti[0], 0.0, 8.0 * ug_fb * sqrt((double)m), s);
            Orth o1{1, 0, false};
            o1.nchol = 1;
            const bool cap = capped(m);
            double lb = cap ? 0.0 : sigma_lb(m, o1);
            CholStatus hs0 = read_st(s);
            const double noise = 16.0 * ug_fb * sqrt((double)m) * hs0.trace;
            const double lb2 = lb * lb - noise;
            if (!cap && lb > 0.0 && lb2 > 4.0 * eps * eps) {
                c->stats.certified_bonds++;
                absorb_next(k, m, X, b, 0);
                fill_identity<T>(*c, m, core[k], m);
                r[k + 1] = m;
                return;
            }
            c->stats.svd_calls++;
            // FP32 data: columns of X = rows of X^T (b x m, in Tmp)
            if constexpr (sizeof(T) == 4) {
                transpose<T>(*c, b, m, X, Tmp);
                if (trunc_f32(m, m, b, Tmp, m, X, eps, k, NR, false)) return;
            }
            jacobi_svd<T>(*c, m, b, X, Ub, SVt, sig, (T*)jwork, svd_tol(b), svd_floor(b));
            std::vector<double> hsg(m);
            TT_CUDA(cudaMemcpyAsync(hsg.data(), sig, m * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
            c->sync();
            const int rp = trunc_rank(hsg, eps);
            // core_k <- U[:, :rp] (m x rp)
            TT_CUDA(cudaMemcpy2DAsync(core[k], rp * sizeof(T), Ub, m * sizeof(T), rp * sizeof(T), m,
                                      cudaMemcpyDeviceToDevice, c->stream));
            absorb_next(k, rp, SVt, b, 0);
            r[k + 1] = rp;
        }
    }

    void lr_sweep(double eps) {
        for (int k = 0; k + 1 < d; ++k) {
            if (k > 0) stream_core(k - 1);  // final since the last iteration
            lr_bond(k, eps);
        }
        if (d >= 2) stream_core(d - 2);
        stream_core(d - 1);
    }

    // ---- pipelined sweeps ------------------------------------------------
    // With second passes skippable (series on, positive budget), a bond is
    // run on the assumption that its first Cholesky QR pass is healthy and
    // its second pass will be skipped (every bond of a well-conditioned
    // rounding): the factor L1 is absorbed into the neighbouring core as
    // soon as the Cholesky ends, on the critical stream, while the apply
    // Q1 = L1^{-1} X, the second Gram, E (and, left to right, the
    // certificate's norms) run on the second stream.  The host reads a
    // bond's decision data after the next bond is queued, so neither the
    // applies nor the host round trip sit on the chain Gram -> Cholesky ->
    // absorb -> next Gram.  A bond that does not pass (unhealthy, E too
    // large for the budget, not certified) is undone with the next one:
    // both streams drain, the cores return to the buffers they started from
    // (the speculative products went to fresh buffers) and the bond runs
    // the sequential path.  The arithmetic of a passed bond is that of the
    // sequential path's skip.
    bool pipe = false;
    bool side_used = false;
    bool tail_used = false;
    bool crit2_used = false;
    static constexpr int kDepth = 3;          // bonds in flight (queued, undecided)
    static constexpr int kPool = 2 * kDepth;  // two fresh core buffers per bond in flight
    std::vector<T*> freeb;                    // free core buffers of the pipeline
    // per slot (bond index mod kDepth): factor, inverse, second Gram, E, L^T
    T *Lq[kDepth] = {}, *Tq[kDepth] = {}, *Gq[kDepth] = {}, *Eq[kDepth] = {}, *Rq[kDepth] = {};
    double* dq = nullptr;                     // device words, 8 per slot
    struct HostSlot {
        CholStatus st;
        double w[4];
    };
    HostSlot* hw = nullptr;  // page-locked mirror of each slot's decision data
    struct Spec {
        int k = -1, slot = 0;
        T *x_orig = nullptr, *q = nullptr;         // core k before; Q1
        T *nb_orig = nullptr, *nb_new = nullptr;  // neighbour before; with L1 absorbed
        CholStatus* s0 = nullptr;
        cudaEvent_t ev_mark = nullptr;  // before the bond's first tile kernel
        cudaEvent_t ev_tail = nullptr;  // after its inverse's tail (tail stream)
        cudaEvent_t ev_col = nullptr;   // before the last tile kernel of a blocked factorization
        cudaEvent_t ev_p0 = nullptr;    // after the absorb's first part (crit2 stream)
        int split = 0;                  // L's columns final at ev_col (0: not blocked)
        cudaEvent_t ev_main = nullptr;  // after the absorb
        cudaEvent_t ev_dec = nullptr;   // after the checks' copies to the host
        bool side_queued = false;
    };
    T* take() {
        if (freeb.empty()) throw_status(TT_ERR_ARG, "internal: pipeline buffers exhausted");
        T* b = freeb.back();
        freeb.pop_back();
        return b;
    }
    void give(T* b) { freeb.push_back(b); }
    void drop_events(Spec& s) {
        for (cudaEvent_t* e : {&s.ev_mark, &s.ev_tail, &s.ev_col, &s.ev_p0, &s.ev_main, &s.ev_dec})
            if (*e) {
                c->ev_pool.push_back(*e);
                *e = nullptr;
            }
    }
    // the bond's factorization, marking the point before its first tile
    // kernel; a blocked factorization leaves its inverse's off-diagonal
    // blocks to the tail stream (only the second stream's work reads them)
    void chol_marked(Spec& s, int a, const T* Gm) {
        s.s0 = next_st();
        s.ev_mark = c->event();
        struct Unmark {
            Ctx* c;
            ~Unmark() {
                c->chol_mark = nullptr;
                c->chol_tail = nullptr;
                c->chol_mark2 = nullptr;
            }
        } um{c};
        c->chol_mark = s.ev_mark;
        c->chol_tail = c->tail();
        s.ev_col = c->event();
        c->chol_mark2 = s.ev_col;
        c->chol_split = 0;
        tail_used = true;
        chol_inv<T, T>(*c, a, Gm, Lq[s.slot], Tq[s.slot], 0.0, 8.0 * ug_fb * sqrt((double)a), s.s0);
        s.split = c->chol_split;
        s.ev_tail = c->event();
        TT_CUDA(cudaEventRecord(s.ev_tail, c->tail()));
    }

    // launches go to the crit2 stream while alive
    struct OnCrit2 {
        Ctx* c;
        cudaStream_t saved;
        explicit OnCrit2(Ctx* cc) : c(cc), saved(cc->stream) { c->stream = c->crit2(); }
        ~OnCrit2() { c->stream = saved; }
    };
    // the point before the bond's last tile kernel (its only one when the
    // factorization is a single tile)
    static cudaEvent_t last_mark(const Spec& s) { return s.split > 0 ? s.ev_col : s.ev_mark; }

    // The absorb of a blocked factorization in two parts: the columns (RL)
    // or rows (LR) left of its last block, which need only L's columns
    // there, on the crit2 stream from the moment they are final (beside the
    // last tile kernel), then the rest on the critical stream, which then
    // waits for the first part.  rl: Y = X L with X
    // (M x a); !rl: Z = L^T C with C (a x NR).
    void split_absorb(Spec& s, bool rl, int M, int a, long NR, const T* X, T* Y) {
        const int p = s.split;
        const T* L = Lq[s.slot];
        {
            OnCrit2 o(c);
            crit2_used = true;
            TT_CUDA(cudaStreamWaitEvent(c->stream, s.ev_col, 0));
            if (rl) mm(false, false, M, p, a, X, a, L, a, Y, a, TRI_B_LOWER, true);
            else mm(true, false, p, (int)NR, a, L, a, X, NR, Y, NR, TRI_A_UPPER, true);
            s.ev_p0 = c->event();
            TT_CUDA(cudaEventRecord(s.ev_p0, c->stream));
        }
        const int q = a - p;
        if (rl) mm(false, false, M, q, q, X + p, a, L + (long)p * a + p, a, Y + p, a, TRI_B_LOWER, true);
        else mm(true, false, q, (int)NR, q, L + (long)p * a + p, a, X + (long)p * NR, NR, Y + (long)p * NR, NR,
                TRI_A_UPPER, true);
        TT_CUDA(cudaStreamWaitEvent(c->stream, s.ev_p0, 0));
    }
    // launches go to the second stream while alive
    struct OnSide {
        Ctx* c;
        cudaStream_t saved;
        explicit OnSide(Ctx* cc) : c(cc), saved(cc->stream) { c->stream = c->side(); }
        ~OnSide() { c->stream = saved; }
    };
    // the critical stream waits for everything queued on the second, tail
    // and crit2 streams
    void join_side() {
        for (int i = 0; i < 3; ++i) {
            if (!(i == 0 ? side_used : i == 1 ? tail_used : crit2_used)) continue;
            cudaEvent_t e = c->event();
            TT_CUDA(cudaEventRecord(e, i == 0 ? c->side() : i == 1 ? c->tail() : c->crit2()));
            TT_CUDA(cudaStreamWaitEvent(c->stream, e, 0));
            c->ev_pool.push_back(e);
        }
    }
    // Q = L1^{-1} X (rows) or X L1^{-T} (cols), as apply_factor does it
    void side_apply(bool rows, int a, long K, const T* X, T* Q, int slot) {
        if constexpr (sizeof(T) == 8) {
            trsm_lower<T>(*c, rows, a, K, Lq[slot], X, Q);
        } else {
            if (rows) mm(false, false, a, (int)K, a, Tq[slot], a, X, K, Q, K, TRI_A_LOWER);
            else mm(false, true, (int)K, a, a, X, a, Tq[slot], a, Q, a, TRI_B_UPPER);
        }
    }
    // (second stream) the bond's status and words to the host, then its event
    void post(Spec& s) {
        TT_CUDA(cudaMemcpyAsync(&hw[s.slot].st, s.s0, sizeof(CholStatus), cudaMemcpyDeviceToHost, c->stream));
        TT_CUDA(cudaMemcpyAsync(hw[s.slot].w, dq + 8 * s.slot, 4 * sizeof(double), cudaMemcpyDeviceToHost,
                                c->stream));
        s.ev_dec = c->event();
        TT_CUDA(cudaEventRecord(s.ev_dec, c->stream));
        s.side_queued = true;
    }
    // the first pass's health and ||E||_F of a bond whose data has arrived
    bool first_pass_ok(const Spec& s, double& e) {
        TT_CUDA(cudaEventSynchronize(s.ev_dec));
        c->stats.host_syncs++;
        const CholStatus h = hw[s.slot].st;
        if (h.nonfinite) throw_status(TT_ERR_NONFINITE, "NaN or Inf in a Gram matrix");
        e = sqrt(hw[s.slot].w[2]);
        const double ratio_fast = tc ? 10.0 * ug_fast : 100.0 * ug_fast;
        return h.ndrop == 0 && h.min_ratio >= ratio_fast && series_valid(e) && e <= skip_budget;
    }
    // returns the events of bonds still queued when a sweep is left by an
    // exception (a normal exit leaves none)
    struct EventGuard {
        Rounder* R;
        std::deque<Spec>* fl;
        ~EventGuard() {
            for (Spec& s : *fl) R->drop_events(s);
        }
    };

    // every stream drains and the pending bonds are undone, newest first:
    // the cores return to the buffers the oldest one started from
    void rollback_all(std::deque<Spec>& fl, bool rl) {
        join_side();
        c->sync();
        for (auto it = fl.rbegin(); it != fl.rend(); ++it) {
            Spec& s = *it;
            core[rl ? s.k - 1 : s.k + 1] = s.nb_orig;
            core[s.k] = s.x_orig;  // the previous pending bond's nb_new
            give(s.q);
            give(s.nb_new);
            drop_events(s);
        }
        fl.clear();
    }

    // The critical stream's part of bond k: Gram, Cholesky, absorb into
    // core k-1 (a fresh buffer)
    Spec main_rl(int k) {
        await_core(k);
        await_core(k - 1);
        Spec s;
        s.k = k;
        s.slot = k % kDepth;
        const int a = r[k];
        const long K = (long)n[k] * r[k + 1];
        const int M = r[k - 1] * n[k - 1];
        s.x_orig = core[k];
        s.nb_orig = core[k - 1];
        s.q = take();
        s.nb_new = take();
        gram_into(true, true, a, K, core[k]);
        chol_marked(s, a, G);
        if (s.split > 0 && s.split < a) split_absorb(s, true, M, a, 0, core[k - 1], s.nb_new);
        else mm(false, false, M, a, a, core[k - 1], a, Lq[s.slot], a, s.nb_new, a, TRI_B_LOWER, true);
        s.ev_main = c->event();
        TT_CUDA(cudaEventRecord(s.ev_main, c->stream));
        core[k - 1] = s.nb_new;
        return s;
    }

    // The second stream's part of bond s.k: Q1 released by `after1`, its
    // Gram, E and the host copies by `after2` (the next bond's first and
    // last tile kernels, so that each of those holds its SM before this
    // work fills the GPU; s's own absorb when no bond follows)
    void side_rl(Spec& s, cudaEvent_t after1, cudaEvent_t after2) {
        const int k = s.k, a = r[k];
        const long K = (long)n[k] * r[k + 1];
        OnSide os(c);
        side_used = true;
        TT_CUDA(cudaStreamWaitEvent(c->stream, after1, 0));
        TT_CUDA(cudaStreamWaitEvent(c->stream, s.ev_tail, 0));
        side_apply(true, a, K, s.x_orig, s.q, s.slot);
        TT_CUDA(cudaStreamWaitEvent(c->stream, after2, 0));
        gram_into(true, K >= kTc2MinK, a, K, s.q, Gq[s.slot]);
        near_identity<T>(*c, a, Gq[s.slot], Eq[s.slot], dq + 8 * s.slot + 2);
        post(s);
    }

    bool resolve_rl(Spec& s) {
        double e = 0.0;
        const bool ok = first_pass_ok(s, e);
        if (!ok) return false;
        skip_budget -= e;
        c->stats.second_pass_skips++;
        core[s.k] = s.q;
        give(s.x_orig);
        give(s.nb_orig);
        drop_events(s);
        return true;
    }


    // Bond k's checks are queued after bond k-1's critical part; the host
    // reads them once bond k-2's critical part is queued too, so it waits
    // for data that arrived a bond earlier while the GPU has two bonds of
    // critical work ahead of it
    void rl_sweep_pipelined() {
        std::deque<Spec> fl;  // bonds queued, not yet decided (oldest first)
        EventGuard eg{this, &fl};
        int k = d - 1;
        for (;;) {
            const bool spec = k >= 1 && (long)n[k] * r[k + 1] > r[k];
            if (spec) {
                Spec cur = main_rl(k);
                if (!fl.empty()) side_rl(fl.back(), cur.ev_mark, last_mark(cur));
                fl.push_back(cur);
                --k;
                if ((int)fl.size() < kDepth) continue;
            } else if (!fl.empty() && !fl.back().side_queued) {
                side_rl(fl.back(), fl.back().ev_main, fl.back().ev_main);
            }
            if (fl.empty()) {
                if (k < 1) break;
                rl_bond(k);  // a rank-cap bond, nothing pending
                --k;
                continue;
            }
            const Spec old = fl.front();
            if (resolve_rl(fl.front())) {
                fl.pop_front();
                continue;
            }
            rollback_all(fl, true);
            rl_bond(old.k);
            k = old.k - 1;  // the bonds after it again, from the corrected cores
        }
        join_side();
    }

    Spec main_lr(int k) {
        Spec s;
        s.k = k;
        s.slot = k % kDepth;
        const int m = r[k] * n[k];
        const int b = r[k + 1];
        s.x_orig = core[k];
        s.nb_orig = core[k + 1];
        s.q = take();
        s.nb_new = take();
        gram_into(false, true, b, m, core[k]);
        chol_marked(s, b, G);
        // core k+1 <- L1^T core k+1
        if (s.split > 0 && s.split < b) {
            split_absorb(s, false, 0, b, (long)n[k + 1] * r[k + 2], core[k + 1], s.nb_new);
            core[k + 1] = s.nb_new;
        } else {
            transpose<T>(*c, b, b, Lq[s.slot], Rq[s.slot]);
            absorb_next(k, b, Rq[s.slot], b, TRI_A_UPPER, s.nb_new);
        }
        s.ev_main = c->event();
        TT_CUDA(cudaEventRecord(s.ev_main, c->stream));
        return s;
    }

    void side_lr(Spec& s, cudaEvent_t after1, cudaEvent_t after2) {
        const int k = s.k, m = r[k] * n[k], b = r[k + 1];
        OnSide os(c);
        side_used = true;
        TT_CUDA(cudaStreamWaitEvent(c->stream, after1, 0));
        TT_CUDA(cudaStreamWaitEvent(c->stream, s.ev_tail, 0));
        side_apply(false, b, m, s.x_orig, s.q, s.slot);
        TT_CUDA(cudaStreamWaitEvent(c->stream, after2, 0));
        gram_into(false, m >= kTc2MinK, b, m, s.q, Gq[s.slot]);
        near_identity<T>(*c, b, Gq[s.slot], Eq[s.slot], dq + 8 * s.slot + 2);
        TT_CUDA(cudaMemsetAsync(dq + 8 * s.slot, 0, 2 * sizeof(double), c->stream));
        inv_and_identity_defect<T>(*c, b, Lq[s.slot], Tq[s.slot], dq + 8 * s.slot);
        post(s);
    }

    // the certified skip of the sequential path (lr_bond with a series
    // pass pending): sigma_min(Q1 L1^T) bounded from L1, its inverse and E
    bool resolve_lr(Spec& s, double eps) {
        double e = 0.0;
        if (!first_pass_ok(s, e)) return false;
        const int b = r[s.k + 1];
        const double sq = sqrt((double)b);
        const double w0 = hw[s.slot].w[0], w1 = hw[s.slot].w[1];
        const double lb1 = std::max(w0 > 0.0 ? 1.0 / sqrt(w0) : 0.0, 1.0 - sqrt(w1));
        const double lb = lb1 * std::max(0.0, sqrt(1.0 - e) - (2.0 + sq) * ug_fb);
        if (!(lb > 2.0 * eps && lb > 0.0)) return false;
        skip_budget -= e;
        c->stats.certified_bonds++;
        c->stats.second_pass_skips++;
        core[s.k] = s.q;
        give(s.x_orig);
        give(s.nb_orig);
        drop_events(s);
        stream_core(s.k, true);
        return true;
    }


    // eps_per_norm: the threshold over ||x|| (delta / sqrt(d - 1)); ||x|| is
    // read at the first decision that needs it (norm_async before)
    void lr_sweep_pipelined(double eps_per_norm) {
        auto eps = [&]() { return eps_per_norm * norm_value(); };
        std::deque<Spec> fl;  // bonds queued, not yet decided (oldest first)
        EventGuard eg{this, &fl};
        int k = 0;
        for (;;) {
            const bool spec = k + 1 < d && r[k] * n[k] >= r[k + 1] && !capped(r[k + 1]) && !pend[k + 1];
            if (spec) {
                Spec cur = main_lr(k);
                if (!fl.empty()) side_lr(fl.back(), cur.ev_mark, last_mark(cur));
                fl.push_back(cur);
                ++k;
                if ((int)fl.size() < kDepth) continue;
            } else if (!fl.empty() && !fl.back().side_queued) {
                side_lr(fl.back(), fl.back().ev_main, fl.back().ev_main);
            }
            if (fl.empty()) {
                if (k + 1 >= d) break;
                lr_bond(k, eps());  // nothing pending: the sequential path
                stream_core(k);
                ++k;
                continue;
            }
            const Spec old = fl.front();
            if (resolve_lr(fl.front(), eps())) {
                fl.pop_front();
                continue;
            }
            rollback_all(fl, false);
            lr_bond(old.k, eps());
            stream_core(old.k);
            k = old.k + 1;
        }
        join_side();
        stream_core(d - 1);
    }

    // one synchronization: the device wait flag (tensor-core and Jacobi
    // kernels), every factorization status of this rounding and the largest
    // ||E||_F of its series passes; false when a series pass was outside
    // its validity (the caller redoes the rounding without them)
    bool check_all_status() {
        std::vector<CholStatus> hs(nst);
        int flag = 0;
        double e2max = 0.0;
        TT_CUDA(cudaMemcpyAsync(&flag, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        if (nst)
            TT_CUDA(cudaMemcpyAsync(hs.data(), st, nst * sizeof(CholStatus), cudaMemcpyDeviceToHost, c->stream));
        if (series_used)
            TT_CUDA(cudaMemcpyAsync(&e2max, dsc + 11, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        c->sync();
        if (flag) {
            TT_CUDA(cudaMemsetAsync(c->tc_err, 0, sizeof(int), c->stream));
            throw_status(TT_ERR_TIMEOUT, "a bounded device wait ran out");
        }
        for (auto& h : hs)
            if (h.nonfinite) throw_status(TT_ERR_NONFINITE, "NaN or Inf in a Gram matrix");
        if (!std::isfinite(e2max)) throw_status(TT_ERR_NONFINITE, "NaN or Inf in a Gram matrix");
        return !series_used || (series_valid(sqrt(e2max)) && !c->series_force_retry);
    }

    tt_tensor* emit() {
        tt_tensor* y = new_tensor(c, d, n.data(), r.data());
        for (int k = 0; k < d; ++k)
            TT_CUDA(cudaMemcpyAsync(y->cores[k], core[k], sizeof(T) * y->core_elems(k), cudaMemcpyDeviceToDevice,
                                    c->stream));
        return y;
    }
};

template <class T>
tt_tensor* finish_round(Rounder<T>& R, const tt_tensor* x, double nrm, double* err_est) {
    tt_tensor* y = R.emit();
    if (sizeof(T) == 8) {
        // FP64: cores 1..d-1 are left-orthonormal to working accuracy, so
        // ||x~|| = ||core_d||_F.  FP32 storage leaves an orthogonality defect
        // of order 1e-6 there; those norms are recomputed on demand with FP64
        // accumulation (norm_internal).
        try {
            y->norm_hint = R.core_norm(x->d - 1);
        } catch (...) {
            free_tensor(y);
            throw;
        }
    }
    if (err_est) *err_est = nrm > 0 ? sqrt(R.err2) / nrm : 0.0;
    return y;
}

// While alive (and on), the context's launches go to its high-priority
// critical stream, which first waits for the caller's stream; on exit the
// caller's stream waits for it.
struct OnCritStream {
    Ctx* c;
    cudaStream_t saved = nullptr;
    bool on = false;
    OnCritStream(Ctx* ctx, bool use) : c(ctx) {
        if (!use) return;
        cudaStream_t crit = c->crit();
        cudaEvent_t e = c->event();
        TT_CUDA(cudaEventRecord(e, c->stream));
        TT_CUDA(cudaStreamWaitEvent(crit, e, 0));
        c->ev_pool.push_back(e);
        saved = c->stream;
        c->stream = crit;
        on = true;
    }
    ~OnCritStream() {
        if (!on) return;
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) {
            cudaEventRecord(e, c->stream);
            cudaStreamWaitEvent(saved, e, 0);
            cudaEventDestroy(e);
        } else {
            cudaStreamSynchronize(c->stream);
        }
        c->stream = saved;
    }
};

template <class T>
tt_tensor* round_t(tt_ctx* ctx, const tt_tensor* x, double delta, double* err_est, void* const* host_out = nullptr,
                   int max_rank = 0, bool fb32_ok = false) {
    ctx->stats.roundings++;
    if (x->d == 1) {
        if (err_est) *err_est = 0.0;
        tt_tensor* y = copy_tensor(ctx, x);
        if (host_out)
            TT_CUDA(cudaMemcpyAsync(host_out[0], y->cores[0], sizeof(T) * y->core_elems(0), cudaMemcpyDeviceToHost,
                                    ctx->stream));
        return y;
    }
    for (int attempt = 0;; ++attempt) {
        // pipelined sweeps on a root context (lanes already overlap whole
        // roundings), not while every kernel family is being timed (each
        // launch is then timed alone; timing one family times its launches
        // where they run), and only where second passes may be skipped; the
        // sweeps then run on the context's critical stream, ordered after
        // and before the caller's
        const bool pipe = attempt == 0 && pipeline_on(ctx);
        OnCritStream cs(ctx, pipe);
        std::unique_ptr<Rounder<T>> Rp;
        try {
            Rp.reset(new Rounder<T>(ctx, x, pipe));
        } catch (const Error& e) {
            // a budget that holds the sequential workspace but not the
            // pipeline's buffers: the sequential sweeps
            if (!pipe || e.status != TT_ERR_OOM) throw;
            Rp.reset(new Rounder<T>(ctx, x, false));
        }
        Rounder<T>& R = *Rp;
        R.host_out = host_out;
        R.max_rank = max_rank;
        R.fb32_ok = fb32_ok;
        if (attempt > 0) R.series = false;
        // skipped second passes (either sweep) leave cores orthonormal to
        // their ||E||_F; the norm and every truncation then see singular
        // values within 1 +- (sum of skipped ||E||_F) / 2, which moves the
        // rounding bound by at most delta times that sum: kept well below
        // the storage precision's resolution of the result, and within 2.5%
        R.skip_budget = (ctx->series_no_skip || ctx->series_force_retry) ? 0.0
                                            : std::min(0.05, (sizeof(T) == 8 ? 1e-14 : 1e-7) / std::max(delta, 1e-300));
        R.rl_sweep();
        double nrm;
        if (R.pipe && R.series && R.skip_budget > 0.0) {
            // ||x|| = ||core_1||_F, read by the host only where the
            // left-to-right sweep first needs its threshold (the sweep's
            // first bonds are queued meanwhile)
            R.norm_async(0);
            R.lr_sweep_pipelined(delta / sqrt((double)(x->d - 1)));
            nrm = R.norm_value();
        } else {
            nrm = R.core_norm(0);
            R.lr_sweep(delta * nrm / sqrt((double)(x->d - 1)));
        }
        if (!R.check_all_status()) {
            // a series pass met a Gram too far from I: redo with Cholesky passes
            ctx->stats.series_retries++;
            continue;
        }
        return finish_round(R, x, nrm, err_est);
    }
}

template <class T>
double norm_t(tt_ctx* ctx, const tt_tensor* x) {
    if (x->d == 1) {
        Rounder<T> R(ctx, x);
        return R.core_norm(0);
    }
    Rounder<T> R(ctx, x);
    R.rl_sweep();
    if (!R.check_all_status()) {
        ctx->stats.series_retries++;
        Rounder<T> R2(ctx, x);
        R2.series = false;
        R2.rl_sweep();
        R2.check_all_status();
        return R2.core_norm(0);
    }
    return R.core_norm(0);
}

}  // namespace

// whether a rounding on this context runs the pipelined sweeps (the
// retries after an invalid series pass never do)
bool pipeline_on(const Ctx* ctx) {
    const Ctx* root = ctx->root ? ctx->root : ctx;
    if (!root->pipeline || (ctx->root && !root->lane_pipeline)) return false;
    return !(ctx->prof && ctx->prof_only.empty()) && ctx->use_series && !ctx->series_no_skip &&
           !ctx->series_force_retry;
}

size_t round_footprint(const tt_tensor* x, tt_precision prec, bool pipelined) {
    const size_t es = prec == TT_FP64 ? 8 : 4;
    int rmax = 1;
    size_t cap = 1, out = 0;
    for (int k = 0; k <= x->d; ++k) rmax = std::max(rmax, x->r[k]);
    for (int k = 0; k < x->d; ++k) {
        cap = std::max(cap, x->core_elems(k));
        out += (x->core_elems(k) * es + 255) & ~size_t(255);  // ranks never grow
    }
    const size_t ws = es == 8 ? Rounder<double>::workspace_bytes(x->d, rmax, cap, es, pipelined)
                              : Rounder<float>::workspace_bytes(x->d, rmax, cap, es, pipelined) +
                                    Rounder<float>::fallback64_bytes(rmax, cap);
    return ws + out;
}

tt_tensor* round_internal(tt_ctx* ctx, const tt_tensor* x, double delta, double* err_est, void* const* host_out,
                          int max_rank, bool fb32_ok) {
    check_tensor(ctx, x);
    if (!(delta >= 0.0) || !isfinite(delta)) throw_status(TT_ERR_ARG, "delta must be finite and >= 0");
    if (max_rank < 0) throw_status(TT_ERR_ARG, "max_rank must be >= 0");
    if (ctx->prec == TT_FP64) return round_t<double>(ctx, x, delta, err_est, host_out, max_rank);
    return round_t<float>(ctx, x, delta, err_est, host_out, max_rank, fb32_ok);
}

double norm_internal(tt_ctx* ctx, const tt_tensor* x) {
    check_tensor(ctx, x);
    if (x->norm_hint >= 0.0) return x->norm_hint;
    if (ctx->prec == TT_FP64) return norm_t<double>(ctx, x);
    // FP32 storage: sqrt(<x, x>) with FP64 accumulation over the stored cores
    double v = 0.0;
    const tt_tensor* ys[1] = {x};
    dot_many_internal(ctx, x, 1, ys, &v);
    if (!isfinite(v)) throw_status(TT_ERR_NONFINITE, "NaN or Inf in the tensor");
    return sqrt(std::max(v, 0.0));
}

}  // namespace ttgb

using namespace ttgb;

extern "C" {

tt_status tt_round(tt_ctx* ctx, const tt_tensor* x, double delta, tt_tensor** out, double* err_est) {
    TT_API_BEGIN
    if (!ctx || !out) throw_status(TT_ERR_ARG, "NULL argument");
    *out = nullptr;
    *out = round_internal(ctx, x, delta, err_est);
    TT_API_END
}

tt_status tt_round_capped(tt_ctx* ctx, const tt_tensor* x, double delta, int max_rank, tt_tensor** out,
                          double* err_est) {
    TT_API_BEGIN
    if (!ctx || !out) throw_status(TT_ERR_ARG, "NULL argument");
    *out = nullptr;
    *out = round_internal(ctx, x, delta, err_est, nullptr, max_rank);
    TT_API_END
}

tt_status tt_round_to_host(tt_ctx* ctx, const tt_tensor* x, double delta, tt_tensor** out, double* err_est,
                           void* const* host_cores) {
    TT_API_BEGIN
    if (!ctx || !out || !host_cores) throw_status(TT_ERR_ARG, "NULL argument");
    *out = nullptr;
    check_tensor(ctx, x);
    for (int k = 0; k < x->d; ++k)
        if (!host_cores[k]) throw_status(TT_ERR_ARG, "NULL host core");
    tt_tensor* y = round_internal(ctx, x, delta, err_est, host_cores);
    try {
        ctx->sync();  // the d = 1 copy runs on the context's stream
    } catch (...) {
        free_tensor(y);
        throw;
    }
    *out = y;
    TT_API_END
}

tt_status tt_norm(tt_ctx* ctx, const tt_tensor* x, double* out) {
    TT_API_BEGIN
    if (!ctx || !out) throw_status(TT_ERR_ARG, "NULL argument");
    *out = norm_internal(ctx, x);
    TT_API_END
}

}  // extern "C"
