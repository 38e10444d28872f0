// Allocation-free TT inner product for callers that must not allocate device
// memory: a host that has already handed all device memory to its own pool
// (a library allocation would fail or break its accounting), or a real-time
// loop where cudaMalloc's implicit device synchronization is not acceptable.
//
// The contraction W_k = sum_i X_k(i)^T W_{k-1} Y_k(i) needs two work arrays
// (W and V); here they live in one file-scope device array of fixed size,
// so the call allocates nothing.  The array is created when the library is
// loaded and every GPU that loads the library holds it until the process
// exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "internal.h"

namespace ttgb {

void set_last_error(const std::string& s);

namespace {

// 1 Mi doubles = 8 MiB per device
constexpr long NOALLOC_ELEMS = 1L << 20;
static __device__ __align__(256) double g_dot_scratch[NOALLOC_ELEMS];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double* g_scratch_ptr[MAX_DEVICES] = {};
int g_sm_count[MAX_DEVICES] = {};

// Device address of the scratch array on the current device, and that
// device's SM count (the GEMMs size their grids by it).  The array's name
// is only a host-side stand-in in host code, so the address is looked up
// once per device with that device current.
double* scratch_for_current_device(int* sm_count) {
    int dev = -1;
    TT_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) throw_status(TT_ERR_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        int sms = 0;
        TT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        TT_CUDA(cudaGetSymbolAddress(&p, g_dot_scratch));
        g_sm_count[dev] = sms;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *sm_count = g_sm_count[dev];
    return g_scratch_ptr[dev];
}

}  // namespace

}  // namespace ttgb

using namespace ttgb;

extern "C" tt_status tt_dot_f64_noalloc(void* cuda_stream, int d, const int* n, const int* rx, const int* ry,
                                        const double* const* x_cores, const double* const* y_cores,
                                        double* result_dev) {
    try {
        if (d < 1 || !n || !rx || !ry || !x_cores || !y_cores || !result_dev)
            throw_status(TT_ERR_ARG, "tt_dot_f64_noalloc: NULL argument or d < 1");
        if (rx[0] != 1 || ry[0] != 1 || rx[d] != 1 || ry[d] != 1)
            throw_status(TT_ERR_ARG, "tt_dot_f64_noalloc: boundary ranks must be 1");
        long wmax = 1, vmax = 1;
        for (int k = 0; k < d; ++k) {
            if (n[k] < 1 || rx[k + 1] < 1 || ry[k + 1] < 1 || !x_cores[k] || !y_cores[k])
                throw_status(TT_ERR_ARG, "tt_dot_f64_noalloc: bad mode size, rank or core pointer");
            wmax = std::max(wmax, (long)rx[k + 1] * ry[k + 1]);
            vmax = std::max(vmax, (long)rx[k] * n[k] * ry[k + 1]);
        }
        if (wmax + vmax > NOALLOC_ELEMS)
            throw_status(TT_ERR_ARG, "tt_dot_f64_noalloc: W (" + std::to_string(wmax) + ") + V (" +
                                         std::to_string(vmax) + ") doubles exceed the static scratch of " +
                                         std::to_string(NOALLOC_ELEMS) + " doubles");
        int sms = 0;
        double* scratch = scratch_for_current_device(&sms);
        // a context object on the stack: no device memory, profiling off
        Ctx c;
        c.stream = (cudaStream_t)cuda_stream;
        c.sm_count = sms;
        double* W = scratch;
        double* V = scratch + wmax;
        fill_identity<double>(c, 1, W, 1);  // W_0 = 1
        for (int k = 0; k < d; ++k) {
            const int nk = n[k], a = rx[k], a2 = rx[k + 1], b = ry[k], b2 = ry[k + 1];
            // V (a x n b2) = W (a x b) Y_k^R (b x n b2)
            gemm<double>(c, false, false, a, nk * b2, b, 1.0, W, b, y_cores[k], (long)nk * b2, 0.0, V,
                         (long)nk * b2);
            // W' (a2 x b2) = (X_k^L)^T (a2 x a n) V^L (a n x b2)
            double* Wn = (k == d - 1) ? result_dev : W;
            gemm<double>(c, true, false, a2, b2, a * nk, 1.0, x_cores[k], a2, V, b2, 0.0, Wn, b2);
        }
        return TT_OK;
    } catch (const Error& e) {
        set_last_error(e.msg);
        return e.status;
    } catch (...) {
        set_last_error("tt_dot_f64_noalloc: unknown error");
        return TT_ERR_CUDA;
    }
}
