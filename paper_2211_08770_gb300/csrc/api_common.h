// Definitions shared by the host-side translation units of the C ABI.
#pragma once

#include <string>
#include <vector>

#include "internal.h"

struct tt_ctx : public ttgb::Ctx {};

struct tt_tensor {
    tt_ctx* ctx = nullptr;
    int d = 0;
    std::vector<int> n, r;
    tt_dtype dtype = TT_DTYPE_F64;
    std::vector<void*> cores;
    void* block = nullptr;   // owned allocation holding every core
    size_t bytes = 0;
    bool owned = false;
    double norm_hint = -1.0; // ||x|| when known exactly from the producer (>= 0)
    size_t core_elems(int k) const { return (size_t)r[k] * n[k] * r[k + 1]; }
};

namespace ttgb {

void set_last_error(const std::string& s);
size_t dtype_size(tt_dtype t);
tt_dtype storage_of(tt_precision p);
void validate_shape(int d, const int* n, const int* r);
tt_tensor* new_tensor(tt_ctx* ctx, int d, const int* n, const int* r);
void free_tensor(tt_tensor* t);
// drops one reference to a context (deleted with its last reference)
void drop_ctx_ref(tt_ctx* c);
tt_tensor* copy_tensor(tt_ctx* ctx, const tt_tensor* x);
void check_same_modes(const tt_tensor* a, const tt_tensor* b);
void check_tensor(tt_ctx* ctx, const tt_tensor* x);
tt_tensor* tt_add_internal(tt_ctx* ctx, int m, const double* alpha, const tt_tensor* const* x);
tt_tensor* scale_internal(tt_ctx* ctx, const tt_tensor* x, double alpha);
// stacked: FP32 storage may take the stacked FP32 contraction of all pairs
// (FP32 products and chunk sums, FP64 across chunks) instead of the FP64
// contraction of each pair (count >= 2; FP64 storage is unaffected)
void dot_many_internal(tt_ctx* ctx, const tt_tensor* x, int count, const tt_tensor* const* y, double* out,
                       bool stacked = false);
// fb32_ok (FP32 storage): the caller vouches that x does not cancel far
// below the scale of its representation, so the fallback orthogonalizations
// may stay in FP32 (otherwise they run in FP64)
tt_tensor* round_internal(tt_ctx* ctx, const tt_tensor* x, double delta, double* err_est,
                          void* const* host_out = nullptr, int max_rank = 0, bool fb32_ok = false);
double norm_internal(tt_ctx* ctx, const tt_tensor* x);
// moves a tensor made on a lane to its root (see get_lanes)
void rehome(tt_tensor* t, Ctx& root);
// One outer iteration of Algorithms 1-4 (scheme TT_CGS, TT_MGS, TT_CGS2 or
// TT_MGS2) for a against the orthonormal Q[0..k-1]: returns the new basis
// vector; col[0..k] receives R(0..k, k).
// qgram (may be NULL, leading dimension ldg): the Gram matrix of Q, which
// lets the modified schemes take all projections of a pass from one batched
// set of dots (see gs_step).
tt_tensor* orth_step_internal(tt_ctx* ctx, tt_scheme scheme, double delta, tt_round_policy policy,
                              const tt_tensor* a, int k, const tt_tensor* const* Q, double* col, int* nrounds,
                              const double* qgram = nullptr, int ldg = 0);
// device bytes a rounding of x may hold at once: workspace plus output
// device bytes a rounding of x may hold at once (its workspace, with the
// pipeline's buffers when pipelined, and its output)
size_t round_footprint(const tt_tensor* x, tt_precision prec, bool pipelined);
// whether roundings on ctx run the pipelined sweeps
bool pipeline_on(const Ctx* ctx);
void round_batched_internal(tt_ctx* ctx, int count, const tt_tensor* const* x, const double* delta, tt_tensor** out);

// RAII owner for tensors created inside drivers
struct TensorGuard {
    tt_tensor* t = nullptr;
    TensorGuard() = default;
    explicit TensorGuard(tt_tensor* x) : t(x) {}
    TensorGuard(const TensorGuard&) = delete;
    TensorGuard& operator=(const TensorGuard&) = delete;
    TensorGuard(TensorGuard&& o) noexcept : t(o.t) { o.t = nullptr; }
    TensorGuard& operator=(TensorGuard&& o) noexcept {
        if (this != &o) { free_tensor(t); t = o.t; o.t = nullptr; }
        return *this;
    }
    ~TensorGuard() { free_tensor(t); }
    tt_tensor* release() { tt_tensor* x = t; t = nullptr; return x; }
    tt_tensor* get() const { return t; }
    void reset(tt_tensor* x) { free_tensor(t); t = x; }
};

}  // namespace ttgb

#define TT_API_BEGIN try {
#define TT_API_END                                                   \
    }                                                                \
    catch (const ttgb::Error& e__) {                                 \
        ttgb::set_last_error(e__.msg);                               \
        return e__.status;                                           \
    }                                                                \
    catch (const std::bad_alloc&) {                                  \
        ttgb::set_last_error("host allocation failed");              \
        return TT_ERR_OOM;                                           \
    }                                                                \
    catch (...) {                                                    \
        ttgb::set_last_error("unknown error");                       \
        return TT_ERR_CUDA;                                          \
    }                                                                \
    return TT_OK;
