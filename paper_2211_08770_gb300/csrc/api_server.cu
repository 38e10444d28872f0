// Request server: TT-round (Section 2) and single outer iterations of the
// Gram-Schmidt schemes (Algorithms 1-4) served from a queue by worker
// lanes, with admission by device footprint and resident bases.
//
// Each worker owns a lane (child context, own non-blocking stream) and a
// host thread.  Requests are admitted from the queue whenever the sum of
// the footprint bounds of the running requests leaves room (continuous
// batching: a finished request frees its share at once and the next one
// starts without waiting for the others).  The oldest waiting request holds
// a reservation: a younger request may only start beside it (the bounds of
// both fit), so large requests are not starved by small ones.
#include <cuda_runtime.h>
#include <math.h>
#include <time.h>

#include <algorithm>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <vector>

#include "api_common.h"

namespace {

using namespace ttgb;

double mono_now() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

struct Request {
    uint64_t ticket = 0;
    tt_request_kind kind = TT_REQ_ROUND;
    const tt_tensor* x = nullptr;
    double delta = 0.0;
    int basis = -1, k = 0;
    tt_scheme scheme = TT_CGS2;
    size_t bound = 0;          // footprint bound (bytes)
    cudaEvent_t ready = nullptr;
    double t_submit = 0, t_start = 0, t_done = 0;
    bool running = false, done = false;
    tt_status status = TT_OK;
    std::string msg;
    tt_tensor* out = nullptr;
    std::vector<double> coef;
    // the first k vectors of the basis and their Gram matrix, copied when
    // the request is admitted (under the server's mutex): the worker never
    // reads the list of bases, which tt_server_add_basis may grow meanwhile
    std::vector<const tt_tensor*> basis_vecs;
    std::vector<double> basis_gram;  // k x k
};

// a resident basis: its vectors and their Gram matrix <q_i, q_j> (k x k)
struct Basis {
    std::vector<tt_tensor*> q;
    std::vector<double> gram;
};

size_t tensor_bytes(const tt_tensor* x, size_t es) {
    size_t b = 0;
    for (int k = 0; k < x->d; ++k) b += (x->core_elems(k) * es + 255) & ~size_t(255);
    return b;
}

}  // namespace

struct tt_server {
    tt_ctx* root = nullptr;
    std::vector<Ctx*> lanes;
    std::vector<std::thread> workers;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::map<uint64_t, Request*> reqs;
    // a deque: appending a basis moves none of the existing ones
    std::deque<Basis> bases;
    size_t budget = 0, in_use = 0, peak = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    tt_server_stats st{};

    // next request allowed to start (caller holds mu), removed from the queue
    Request* pick() {
        if (queue.empty()) return nullptr;
        Request* head = queue.front();
        if (in_use + head->bound <= budget) {
            queue.pop_front();
            return head;
        }
        for (auto it = queue.begin() + 1; it != queue.end(); ++it) {
            if (in_use + (*it)->bound + head->bound <= budget) {
                Request* r = *it;
                queue.erase(it);
                return r;
            }
        }
        return nullptr;
    }

    // footprint bound of a request (bytes it may hold at once on the device)
    size_t bound_of(const Request& q) const {
        const size_t es = root->prec == TT_FP64 ? 8 : 4;
        const bool pipe = root->pipeline && root->lane_pipeline;
        if (q.kind == TT_REQ_ROUND) return round_footprint(q.x, root->prec, pipe) + (1u << 20);
        // the concatenated sum x - sum_j r_j q_j: ranks add up bond by bond
        const tt_tensor* x = q.x;
        const std::vector<tt_tensor*>& B = bases[q.basis].q;
        std::vector<int> r(x->r);
        for (int j = 0; j < q.k; ++j)
            for (int b = 1; b < x->d; ++b) r[b] += B[j]->r[b];
        tt_tensor S;  // shape only
        S.d = x->d;
        S.n = x->n;
        S.r = r;
        const size_t sb = tensor_bytes(&S, es);
        // the running sum and its successor (MGS), the rounding of the sum,
        // the normalised copy, and FP64 copies for the projections when FP32
        size_t b = 2 * sb + round_footprint(&S, root->prec, pipe) + sb;
        if (es == 4) b += 2 * tensor_bytes(&S, 8);
        // the stacked dots of a pass (x at most the concatenation's ranks)
        size_t wmax = 1, vmax = 1, pmax = 1;
        for (int c = 0; c < x->d; ++c) {
            size_t Sc = 0, Sc2 = 0;
            for (int j = 0; j < q.k; ++j) {
                Sc += B[j]->r[c];
                Sc2 += B[j]->r[c + 1];
            }
            const size_t K = (size_t)r[c] * x->n[c];
            wmax = std::max(wmax, std::max((size_t)r[c] * Sc, (size_t)r[c + 1] * Sc2));
            vmax = std::max(vmax, K * Sc2);
            pmax = std::max(pmax, ((K + 255) / 256) * r[c + 1] * Sc2);
        }
        b += 2 * wmax * 8 + (vmax + pmax) * es;
        return b + (1u << 20);
    }

    void run(Ctx* lane, Request* q) {
        tt_ctx* l = static_cast<tt_ctx*>(lane);
        try {
            TT_CUDA(cudaStreamWaitEvent(lane->stream, q->ready, 0));
            if (q->kind == TT_REQ_ROUND) {
                q->out = round_internal(l, q->x, q->delta, nullptr);
            } else {
                q->coef.assign(q->k + 1, 0.0);
                q->out = orth_step_internal(l, q->scheme, q->delta, TT_ROUND_PAPER, q->x, q->k,
                                            q->basis_vecs.data(), q->coef.data(), nullptr,
                                            q->basis_gram.data(), q->k);
            }
            lane->sync();  // the result is complete on the device
            rehome(q->out, *root);
        } catch (const Error& e) {
            q->status = e.status;
            q->msg = e.msg;
        } catch (const std::bad_alloc&) {
            q->status = TT_ERR_OOM;
            q->msg = "host allocation failed";
        } catch (...) {
            q->status = TT_ERR_CUDA;
            q->msg = "unexpected exception in a server worker";
        }
        if (q->status != TT_OK && q->out) {
            cudaStreamSynchronize(lane->stream);
            if (q->out->ctx != root) rehome(q->out, *root);
            free_tensor(q->out);
            q->out = nullptr;
        }
    }

    void worker(Ctx* lane) {
        cudaSetDevice(lane->device);
        for (;;) {
            Request* q = nullptr;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] { return stop || (q = pick()) != nullptr; });
                if (!q) return;  // stopping and nothing admissible
                in_use += q->bound;
                peak = std::max(peak, in_use);
                q->running = true;
                q->t_start = mono_now();
                if (q->kind == TT_REQ_ORTH_STEP) {
                    const Basis& B = bases[q->basis];
                    const int kb = (int)B.q.size();
                    q->basis_vecs.assign(B.q.begin(), B.q.begin() + q->k);
                    q->basis_gram.resize((size_t)q->k * q->k);
                    for (int i = 0; i < q->k; ++i)
                        for (int j = 0; j < q->k; ++j) q->basis_gram[(size_t)i * q->k + j] = B.gram[(size_t)i * kb + j];
                }
            }
            run(lane, q);
            {
                std::lock_guard<std::mutex> lk(mu);
                q->t_done = mono_now();
                in_use -= q->bound;
                q->running = false;
                q->done = true;
                if (q->status == TT_OK) st.completed++;
                else st.failed++;
                st.roundings += lane->stats.roundings;
                st.kernel_launches += lane->stats.kernel_launches;
                st.host_syncs += lane->stats.host_syncs;
                lane->stats = tt_stats{};
                lane->recs.clear();
            }
            cv_done.notify_all();
            cv_work.notify_all();  // the freed footprint may admit others
        }
    }
};

using namespace ttgb;

extern "C" {

tt_status tt_server_create(tt_ctx* ctx, int workers, size_t footprint_budget, tt_server** out) {
    TT_API_BEGIN
    if (!ctx || !out || ctx->root || workers < 1 || workers > TT_MAX_LANES) throw_status(TT_ERR_ARG, "bad arguments");
    *out = nullptr;
    std::unique_ptr<tt_server> s(new tt_server());
    s->root = ctx;
    s->budget = footprint_budget ? footprint_budget : (ctx->budget ? ctx->budget : SIZE_MAX);
    s->st.footprint_budget = s->budget == SIZE_MAX ? 0 : s->budget;
    // private lanes (not the context's batched-rounding lanes)
    for (int w = 0; w < workers; ++w) {
        Ctx* l = new tt_ctx();
        s->lanes.push_back(l);
        l->device = ctx->device;
        l->root = ctx;
        l->owns_stream = true;
        l->prec = ctx->prec;
        l->sign_rule = ctx->sign_rule;
        l->sm_count = ctx->sm_count;
        l->use_tc = ctx->use_tc;
        l->use_tc_gemm = ctx->use_tc_gemm;
        l->tc_gemm_split = ctx->tc_gemm_split;
        l->tc_wait_limit = ctx->tc_wait_limit;
        l->use_tc_absorb = ctx->use_tc_absorb;
        cudaError_t e = cudaStreamCreateWithFlags(&l->stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMalloc(&l->tc_err, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(l->tc_err, 0, sizeof(int));
        if (e != cudaSuccess) {
            cudaGetLastError();
            for (Ctx* x : s->lanes) delete static_cast<tt_ctx*>(x);
            throw_cuda(e, "server lane creation", __FILE__, __LINE__);
        }
    }
    ctx->refs++;  // the context outlives the server's tensors
    tt_server* raw = s.get();
    try {
        for (Ctx* l : raw->lanes) raw->workers.emplace_back([raw, l] { raw->worker(l); });
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(raw->mu);
            raw->stop = true;
        }
        raw->cv_work.notify_all();
        for (auto& t : raw->workers) t.join();
        for (Ctx* x : raw->lanes) delete static_cast<tt_ctx*>(x);
        drop_ctx_ref(ctx);
        throw_status(TT_ERR_OOM, "could not start the server workers");
    }
    *out = s.release();
    TT_API_END
}

tt_status tt_server_add_basis(tt_server* s, int k, const tt_tensor* const* q, int* basis_id) {
    TT_API_BEGIN
    if (!s || k < 1 || !q || !basis_id) throw_status(TT_ERR_ARG, "bad arguments");
    for (int j = 0; j < k; ++j) {
        check_tensor(s->root, q[j]);
        check_same_modes(q[0], q[j]);
    }
    Basis B;
    try {
        for (int j = 0; j < k; ++j) B.q.push_back(copy_tensor(s->root, q[j]));
        // <q_i, q_j> once per basis: the modified schemes' projections of a
        // step are then formed from one batched set of dots (gs_step)
        B.gram.assign((size_t)k * k, 0.0);
        std::vector<const tt_tensor*> qs(B.q.begin(), B.q.end());
        std::vector<double> row(k);
        for (int i = 0; i < k; ++i) {
            dot_many_internal(s->root, B.q[i], i + 1, qs.data(), row.data(), true);
            for (int j = 0; j <= i; ++j) B.gram[(size_t)i * k + j] = B.gram[(size_t)j * k + i] = row[j];
        }
    } catch (...) {
        for (auto* t : B.q) free_tensor(t);
        throw;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->bases.push_back(std::move(B));
    *basis_id = (int)s->bases.size() - 1;
    TT_API_END
}

tt_status tt_server_submit(tt_server* s, tt_request_kind kind, const tt_tensor* x, double delta, int basis_id,
                           int k, tt_scheme scheme, uint64_t* ticket) {
    TT_API_BEGIN
    if (!s || !ticket) throw_status(TT_ERR_ARG, "bad arguments");
    *ticket = 0;
    check_tensor(s->root, x);
    if (!(delta >= 0.0) || !isfinite(delta)) throw_status(TT_ERR_ARG, "delta must be finite and >= 0");
    std::unique_ptr<Request> q(new Request());
    q->kind = kind;
    q->x = x;
    q->delta = delta;
    if (kind == TT_REQ_ORTH_STEP) {
        if (scheme != TT_CGS && scheme != TT_MGS && scheme != TT_CGS2 && scheme != TT_MGS2)
            throw_status(TT_ERR_ARG, "an orthogonalization step takes TT_CGS, TT_MGS, TT_CGS2 or TT_MGS2");
        std::lock_guard<std::mutex> lk(s->mu);
        if (basis_id < 0 || basis_id >= (int)s->bases.size()) throw_status(TT_ERR_ARG, "unknown basis");
        if (k < 0 || k > (int)s->bases[basis_id].q.size()) throw_status(TT_ERR_ARG, "k exceeds the basis size");
        if (k > 0) check_same_modes(s->bases[basis_id].q[0], x);
        q->basis = basis_id;
        q->k = k;
        q->scheme = scheme;
    } else if (kind != TT_REQ_ROUND) {
        throw_status(TT_ERR_ARG, "bad request kind");
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        q->bound = s->bound_of(*q);
        if (q->bound > s->budget) {
            s->st.refused++;
            throw_status(TT_ERR_OOM, "request footprint bound (" + std::to_string(q->bound) +
                                         " bytes) exceeds the server budget (" + std::to_string(s->budget) + ")");
        }
    }
    TT_CUDA(cudaEventCreateWithFlags(&q->ready, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(q->ready, s->root->stream);
    if (e != cudaSuccess) {
        cudaEventDestroy(q->ready);
        throw_cuda(e, "cudaEventRecord", __FILE__, __LINE__);
    }
    Request* r = q.release();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->ticket = s->next_ticket++;
        r->t_submit = mono_now();
        s->reqs[r->ticket] = r;
        s->queue.push_back(r);
        s->st.submitted++;
        *ticket = r->ticket;
    }
    s->cv_work.notify_one();
    TT_API_END
}

tt_status tt_server_wait(tt_server* s, uint64_t ticket, int timeout_ms, tt_tensor** out, double* coef,
                         int coef_cap, double* times) {
    TT_API_BEGIN
    if (!s || (coef_cap > 0 && !coef)) throw_status(TT_ERR_ARG, "bad arguments");
    if (out) *out = nullptr;
    Request* q = nullptr;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) throw_status(TT_ERR_ARG, "unknown ticket");
        q = it->second;
        auto done = [&] { return q->done; };
        if (timeout_ms < 0) s->cv_done.wait(lk, done);
        else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done))
            throw_status(TT_ERR_TIMEOUT, "request not finished within the timeout");
        s->reqs.erase(it);
    }
    std::unique_ptr<Request> own(q);
    if (q->ready) cudaEventDestroy(q->ready);
    if (times) {
        times[0] = q->t_submit;
        times[1] = q->t_start;
        times[2] = q->t_done;
    }
    for (int j = 0; j < coef_cap && j < (int)q->coef.size(); ++j) coef[j] = q->coef[j];
    if (q->status != TT_OK) throw_status(q->status, q->msg);
    if (out) *out = q->out;
    else free_tensor(q->out);
    TT_API_END
}

tt_status tt_server_cancel(tt_server* s, uint64_t ticket) {
    TT_API_BEGIN
    if (!s) throw_status(TT_ERR_ARG, "bad arguments");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) throw_status(TT_ERR_ARG, "unknown ticket");
        Request* q = it->second;
        auto pos = std::find(s->queue.begin(), s->queue.end(), q);
        if (pos == s->queue.end()) throw_status(TT_ERR_ARG, "the request has started or finished");
        s->queue.erase(pos);
        q->status = TT_ERR_CANCELLED;
        q->msg = "cancelled before it started";
        q->done = true;
        q->t_start = q->t_done = mono_now();
        s->st.cancelled++;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();  // the head's reservation may have gone
    TT_API_END
}

tt_status tt_server_get_stats(tt_server* s, tt_server_stats* out) {
    if (!s || !out) return TT_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    out->queued = s->queue.size();
    uint64_t running = 0;
    for (auto& kv : s->reqs) running += kv.second->running ? 1 : 0;
    out->running = running;
    out->footprint_in_use = s->in_use;
    out->footprint_peak = s->peak;
    return TT_OK;
}

void tt_server_destroy(tt_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (Request* q : s->queue) {
            q->status = TT_ERR_CANCELLED;
            q->done = true;
        }
        s->queue.clear();
        s->stop = true;
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
    for (auto& t : s->workers) t.join();
    for (auto& kv : s->reqs) {
        Request* q = kv.second;
        if (q->ready) cudaEventDestroy(q->ready);
        free_tensor(q->out);
        delete q;
    }
    for (auto& B : s->bases)
        for (auto* t : B.q) free_tensor(t);
    for (Ctx* l : s->lanes) {
        cudaStreamSynchronize(l->stream);
        delete static_cast<tt_ctx*>(l);
    }
    tt_ctx* root = s->root;
    delete s;
    drop_ctx_ref(root);
}

}  // extern "C"
