// Batched TT-rounding: many independent roundings (TT-round of Section 2 applied to
// a list of tensors) run concurrently on lanes, each lane a child context
// with its own non-blocking stream, workspace and host worker thread.
//
// A rounding alternates short kernels with host decisions (pivot health,
// truncation ranks), so one rounding leaves most of the 152 SMs idle and
// the host waits on its stream between phases.  Running L roundings at once
// on L streams overlaps those waits and fills the GPU with the kernels of
// several instances; instances are taken largest-first from a shared
// counter (longest-processing-time order), so the lanes finish together.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <numeric>
#include <thread>
#include <vector>

#include "api_common.h"

namespace ttgb {

std::vector<Ctx*> get_lanes(Ctx& root, int count) {
    while ((int)root.lanes.size() < count) {
        Ctx* l = new tt_ctx();  // deleted by the root's destructor as a tt_ctx
        l->device = root.device;
        l->root = &root;
        l->owns_stream = true;
        cudaError_t e = cudaStreamCreateWithFlags(&l->stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMalloc(&l->tc_err, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(l->tc_err, 0, sizeof(int));
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete l;
            throw_cuda(e, "lane creation", __FILE__, __LINE__);
        }
        root.lanes.push_back(l);
    }
    std::vector<Ctx*> out(root.lanes.begin(), root.lanes.begin() + count);
    for (Ctx* l : out) {  // settings follow the root's current ones
        l->prec = root.prec;
        l->sign_rule = root.sign_rule;
        l->sm_count = root.sm_count;
        l->use_tc = root.use_tc;
        l->use_tc_gemm = root.use_tc_gemm;
        l->tc_gemm_split = root.tc_gemm_split;
        l->tc_wait_limit = root.tc_wait_limit;
        l->use_tc_absorb = root.use_tc_absorb;
        l->chol_nb = root.chol_nb;
        l->colgram_stages = root.colgram_stages;
        l->pipeline = root.pipeline;
        l->use_series = root.use_series;
        l->series_force_retry = root.series_force_retry;
        l->series_no_skip = root.series_no_skip;
        l->prof = root.prof;
        l->prof_only = root.prof_only;
    }
    return out;
}

void merge_lane(Ctx& root, Ctx& lane) {
    root.stats.kernel_launches += lane.stats.kernel_launches;
    root.stats.roundings += lane.stats.roundings;
    root.stats.host_syncs += lane.stats.host_syncs;
    root.stats.svd_calls += lane.stats.svd_calls;
    root.stats.certified_bonds += lane.stats.certified_bonds;
    root.stats.fallback_orth += lane.stats.fallback_orth;
    root.stats.svd_sweeps += lane.stats.svd_sweeps;
    root.stats.series_passes += lane.stats.series_passes;
    root.stats.series_retries += lane.stats.series_retries;
    root.stats.second_pass_skips += lane.stats.second_pass_skips;
    root.stats.fallback_fp32 += lane.stats.fallback_fp32;
    lane.stats = tt_stats{};
    for (auto& r : lane.recs) {
        ProfRec q = r;
        q.fam = root.family(lane.fam_names[r.fam].c_str());
        root.recs.push_back(q);
    }
    lane.recs.clear();
}

void rehome(tt_tensor* t, Ctx& root) {
    Ctx* from = t->ctx;
    if (from == &root) return;
    t->ctx = static_cast<tt_ctx*>(&root);
    root.refs++;
    from->refs--;  // a lane is never deleted by its tensors: its root owns it
}

// Estimated floating-point work of rounding x: the Gram, apply and absorb
// products of both sweeps, ~ sum_k n_k r_{k-1} r_k (r_{k-1} + r_k).
static double rounding_cost(const tt_tensor* x) {
    double s = 0.0;
    for (int k = 0; k < x->d; ++k) {
        double a = x->r[k], b = x->r[k + 1];
        s += x->n[k] * a * b * (a + b);
    }
    return s;
}

void round_batched_internal(tt_ctx* ctx, int count, const tt_tensor* const* x, const double* delta,
                            tt_tensor** out) {
    for (int i = 0; i < count; ++i) {
        check_tensor(ctx, x[i]);
        if (!(delta[i] >= 0.0) || !isfinite(delta[i])) throw_status(TT_ERR_ARG, "delta must be finite and >= 0");
    }
    std::vector<tt_tensor*> res(count, nullptr);
    const int L = std::min(ctx->max_lanes, count);
    if (L <= 1) {
        try {
            for (int i = 0; i < count; ++i) res[i] = round_internal(ctx, x[i], delta[i], nullptr);
        } catch (...) {
            for (auto* t : res) free_tensor(t);
            throw;
        }
        for (int i = 0; i < count; ++i) out[i] = res[i];
        return;
    }
    std::vector<Ctx*> lanes = get_lanes(*ctx, L);
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::vector<double> cost(count);
    for (int i = 0; i < count; ++i) cost[i] = rounding_cost(x[i]);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });

    // inputs were produced on the root's stream: every lane starts after it
    cudaEvent_t ready = ctx->event();
    TT_CUDA(cudaEventRecord(ready, ctx->stream));
    for (Ctx* l : lanes) TT_CUDA(cudaStreamWaitEvent(l->stream, ready, 0));
    ctx->ev_pool.push_back(ready);

    std::atomic<int> next{0};
    std::atomic<bool> abort{false};
    std::mutex emu;
    bool failed = false;
    Error first{TT_OK, ""};
    auto fail = [&](tt_status s, const std::string& m) {
        std::lock_guard<std::mutex> lk(emu);
        if (!failed) {
            failed = true;
            first = Error{s, m};
        }
        abort = true;
    };
    auto work = [&](Ctx* l) {
        try {
            TT_CUDA(cudaSetDevice(l->device));
            while (!abort.load()) {
                const int j = next.fetch_add(1);
                if (j >= count) break;
                const int i = order[j];
                res[i] = round_internal(static_cast<tt_ctx*>(l), x[i], delta[i], nullptr);
            }
        } catch (const Error& e) {
            fail(e.status, e.msg);
        } catch (const std::bad_alloc&) {
            fail(TT_ERR_OOM, "host allocation failed");
        } catch (...) {
            fail(TT_ERR_CUDA, "unexpected exception in a batched-rounding worker");
        }
    };
    std::vector<std::thread> pool;
    pool.reserve(L - 1);
    try {
        for (int w = 1; w < L; ++w) pool.emplace_back(work, lanes[w]);
    } catch (...) {
        abort = true;
        for (auto& t : pool) t.join();
        throw_status(TT_ERR_OOM, "could not start the batched-rounding workers");
    }
    work(lanes[0]);  // the calling thread is lane 0's worker
    for (auto& t : pool) t.join();
    TT_CUDA(cudaSetDevice(ctx->device));

    // the root's stream continues after every lane's last launch
    for (Ctx* l : lanes) {
        cudaEvent_t done = l->event();
        TT_CUDA(cudaEventRecord(done, l->stream));
        TT_CUDA(cudaStreamWaitEvent(ctx->stream, done, 0));
        l->ev_pool.push_back(done);
        merge_lane(*ctx, *l);
    }
    for (auto* t : res)
        if (t) rehome(t, *ctx);
    if (failed) {
        for (auto* t : res) free_tensor(t);
        throw first;
    }
    for (int i = 0; i < count; ++i) out[i] = res[i];
}

}  // namespace ttgb

using namespace ttgb;

extern "C" {

tt_status tt_round_batched(tt_ctx* ctx, int count, const tt_tensor* const* x, const double* delta, tt_tensor** out) {
    TT_API_BEGIN
    if (!ctx || !out || count < 0 || (count > 0 && (!x || !delta))) throw_status(TT_ERR_ARG, "bad arguments");
    for (int i = 0; i < count; ++i) out[i] = nullptr;
    if (count > 0) round_batched_internal(ctx, count, x, delta, out);
    TT_API_END
}

tt_status tt_ctx_set_concurrency(tt_ctx* ctx, int lanes) {
    if (!ctx || ctx->root || lanes < 1 || lanes > TT_MAX_LANES) return TT_ERR_ARG;
    ctx->max_lanes = lanes;
    return TT_OK;
}

int tt_ctx_get_concurrency(const tt_ctx* ctx) { return ctx ? ctx->max_lanes : 0; }

}  // extern "C"
