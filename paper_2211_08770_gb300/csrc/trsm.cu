// Triangular solves with the Cholesky factor for the fallback passes of
// TT-round's orthogonalization: Q = L^{-1} X (the right unfolding's rows)
// or Q = X L^{-T} (the left unfolding's columns), blocked by 32 rows of L.
// Off-diagonal blocks are GEMM updates; each diagonal block is solved by
// forward substitution, one vector per thread with the 32 x 32 block in
// shared memory, in FP64 arithmetic.  Unlike the product with an explicit
// inverse L^{-1} (whose error grows with kappa(L) u), the substitution is
// backward stable: L Q = X + O(u) |L| |Q|, which keeps the content of an
// ill-conditioned unfolding (a sum that cancels far below its terms) that
// the shifted Cholesky QR passes must preserve.  A zero pivot (a dropped
// direction) gives a zero component.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace ttgb {

namespace {

constexpr int NB = 32;

// Q holds the right-hand sides on entry and the solution on return: vector v
// has its element j at Q[j * ldq + v] (ROWS) or Q[v * ldq + j] (!ROWS)
template <class T, bool ROWS>
__global__ void __launch_bounds__(256) trsm_diag_kernel(int nb, const T* __restrict__ Lii, long ldl,
                                                        T* __restrict__ Q, long ldq, long nvec) {
    __shared__ double Ls[NB][NB + 1];
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int r = e / NB, cc = e % NB;
        Ls[r][cc] = (r < nb && cc <= r) ? (double)Lii[(long)r * ldl + cc] : 0.0;
    }
    __syncthreads();
    for (long v = blockIdx.x * (long)blockDim.x + threadIdx.x; v < nvec; v += (long)gridDim.x * blockDim.x) {
        double q[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            double b = 0.0;
            if (j < nb) b = ROWS ? (double)Q[(long)j * ldq + v] : (double)Q[v * ldq + j];
#pragma unroll
            for (int l = 0; l < j; ++l) b -= Ls[j][l] * q[l];
            q[j] = Ls[j][j] != 0.0 ? b / Ls[j][j] : 0.0;
        }
#pragma unroll
        for (int j = 0; j < NB; ++j)
            if (j < nb) {
                if (ROWS) Q[(long)j * ldq + v] = (T)q[j];
                else Q[v * ldq + j] = (T)q[j];
            }
    }
}

unsigned grid_for_vectors(const Ctx& c, long n) {
    const long want = (n + 255) / 256;
    return (unsigned)std::max(1L, std::min(want, (long)std::max(1, c.sm_count) * 8));
}

}  // namespace

// rows: Q (a x K, row-major) = L^{-1} X; !rows: Q (K x a, row-major) =
// X L^{-T}.  L is a x a lower triangular (leading dimension a).  Q may not
// alias X.
template <class T>
void trsm_lower(Ctx& c, bool rows, int a, long K, const T* L, const T* X, T* Q) {
    const size_t nel = (size_t)a * K;
    TT_CUDA(cudaMemcpyAsync(Q, X, nel * sizeof(T), cudaMemcpyDeviceToDevice, c.stream));
    ProfScope ps(c, sizeof(T) == 8 ? "trsm_f64" : "trsm_f32", (double)a * a * (double)K,
                 sizeof(T) * (2.0 * nel + (double)a * a));
    for (int i0 = 0; i0 < a; i0 += NB) {
        const int nb = std::min(NB, a - i0);
        if (rows) {
            // Q_i -= L_{i,<i} Q_{<i}
            if (i0 > 0)
                gemm<T>(c, false, false, nb, (int)K, i0, T(-1), L + (long)i0 * a, a, Q, K, T(1), Q + (long)i0 * K, K);
            trsm_diag_kernel<T, true><<<grid_for_vectors(c, K), 256, 0, c.stream>>>(
                nb, L + (long)i0 * a + i0, a, Q + (long)i0 * K, K, K);
        } else {
            // Q_{:,i} -= Q_{:,<i} L_{i,<i}^T
            if (i0 > 0)
                gemm<T>(c, false, true, (int)K, nb, i0, T(-1), Q, a, L + (long)i0 * a, a, T(1), Q + i0, a);
            trsm_diag_kernel<T, false><<<grid_for_vectors(c, K), 256, 0, c.stream>>>(
                nb, L + (long)i0 * a + i0, a, Q + i0, a, K);
        }
        TT_LAUNCHED(c);
    }
}

template void trsm_lower<double>(Ctx&, bool, int, long, const double*, const double*, double*);
template void trsm_lower<float>(Ctx&, bool, int, long, const float*, const float*, float*);

}  // namespace ttgb
