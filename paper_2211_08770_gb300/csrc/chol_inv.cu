// Blocked Cholesky factorization with rank drop and explicit inverse of the
// factor, one CTA, for the small r x r Gram matrices of the Cholesky QR
// passes of TT-round:  G + s I = L L^T, T = L^{-1}.
//
// Right-looking over 32-column panels: warp 0 factors the 32 x 32 diagonal
// block in shared memory (pivots <= drop threshold are dropped: their column
// of L is zeroed) and inverts it; all warps then solve the panel below it and
// apply the symmetric rank-32 update to the trailing lower triangle, one
// 32 x 32 tile per warp at a time.  The inverse is assembled block row by
// block row, T_IJ = -T_II sum_{K=J}^{I-1} L_IK T_KJ, the J blocks of a row in
// parallel.  The matrices live in global memory (L2-resident at these sizes);
// the tiles a warp works on are staged in its own shared-memory slots.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "internal.h"

namespace ttgb {

namespace {

constexpr unsigned FULL = 0xffffffffu;

template <class C>
__device__ __forceinline__ C wsum(C v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// per-warp staging: Ks (32 x 32, read by broadcast) and Is (32 x 33, read by
// row per lane)
template <class C>
struct WarpTiles {
    C Ks[32][32];
    C Is[32][33];
};

template <class S, class C, int NT>
__global__ void __launch_bounds__(NT)
chol_inv_kernel(int n, const S* __restrict__ G, S* __restrict__ L, S* __restrict__ Tm, double shift_rel,
                double drop_rel, CholStatus* st) {
    extern __shared__ __align__(16) unsigned char ci_smem[];
    constexpr int NW = NT / 32;
    WarpTiles<C>* wt = reinterpret_cast<WarpTiles<C>*>(ci_smem);
    __shared__ C Ds[32][33];
    __shared__ C Di[32][33];
    __shared__ double shd[32];
    __shared__ int s_ndrop, s_nonfinite;
    __shared__ double s_minratio;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // trace and largest diagonal entry of G
    double tr = 0.0, mx = 0.0;
    for (int i = tid; i < n; i += NT) {
        const double g = (double)G[(long)i * n + i];
        tr += g;
        mx = fmax(mx, g);
    }
    tr = wsum(tr);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(FULL, mx, o));
    if (lane == 0) shd[warp] = tr;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < NW; ++w) t += shd[w];
        shd[0] = t;
        s_ndrop = 0;
        s_nonfinite = 0;
        s_minratio = 1e300;
    }
    __syncthreads();
    tr = shd[0];
    __syncthreads();
    if (lane == 0) shd[warp] = mx;
    __syncthreads();
    if (tid == 0) {
        double m = 0.0;
        for (int w = 0; w < NW; ++w) m = fmax(m, shd[w]);
        shd[0] = m;
    }
    __syncthreads();
    mx = shd[0];
    const double shift = shift_rel * tr;
    const double tau = drop_rel * (mx + shift);

    const long nn = (long)n * n;
    for (long e = tid; e < nn; e += NT) {
        const long i = e / n, k = e % n;
        L[e] = (k <= i) ? (S)((C)G[e] + (i == k ? (C)shift : C(0))) : S(0);
        Tm[e] = S(0);
    }
    __syncthreads();

    const int P = (n + 31) / 32;
    for (int p = 0; p < P; ++p) {
        const int j0 = p * 32, jb = min(32, n - j0);
        // (1) diagonal block: factor + inverse by warp 0
        if (warp == 0) {
            for (int k = 0; k < 32; ++k)
                Ds[lane][k] = (lane < jb && k <= lane) ? (C)L[(long)(j0 + lane) * n + j0 + k] : C(0);
            __syncwarp();
            for (int c = 0; c < jb; ++c) {
                const C piv = Ds[c][c];
                const double orig = (double)G[(long)(j0 + c) * n + j0 + c] + shift;
                const bool fin = isfinite((double)piv);
                const bool keep = fin && (double)piv > tau && piv > C(0);
                const C dc = keep ? sqrt(piv) : C(0);
                __syncwarp();
                if (lane == c) Ds[c][c] = dc;
                if (lane > c && lane < jb) Ds[lane][c] = keep ? Ds[lane][c] / dc : C(0);
                __syncwarp();
                if (keep && lane > c && lane < jb) {
                    const C lic = Ds[lane][c];
                    for (int k = c + 1; k <= lane; ++k) Ds[lane][k] -= lic * Ds[k][c];
                }
                if (lane == 0) {
                    if (!fin) s_nonfinite = 1;
                    if (keep) s_minratio = fmin(s_minratio, orig > 0.0 ? (double)piv / orig : 0.0);
                    else s_ndrop++;
                }
                __syncwarp();
            }
            // inverse of the diagonal block: lane j forms column j
            {
                const int j = lane;
                for (int i = 0; i < 32; ++i) Di[i][j] = C(0);
                if (j < jb && Ds[j][j] != C(0)) {
                    Di[j][j] = C(1) / Ds[j][j];
                    for (int i = j + 1; i < jb; ++i) {
                        const C dii = Ds[i][i];
                        if (dii == C(0)) continue;
                        C s = C(0);
                        for (int k = j; k < i; ++k) s += Ds[i][k] * Di[k][j];
                        Di[i][j] = -s / dii;
                    }
                }
            }
            __syncwarp();
            for (int k = 0; k < jb; ++k) {
                if (lane < jb && k <= lane) {
                    L[(long)(j0 + lane) * n + j0 + k] = (S)Ds[lane][k];
                    Tm[(long)(j0 + lane) * n + j0 + k] = (S)Di[lane][k];
                }
            }
        }
        __syncthreads();
        // (2) panel: L[i, panel] = A[i, panel] * L_pp^{-T} for the rows below
        for (int i = j0 + jb + warp; i < n; i += NW) {
            const C a = (lane < jb) ? (C)L[(long)i * n + j0 + lane] : C(0);
            C out = C(0);
            for (int k = 0; k < jb; ++k) out += __shfl_sync(FULL, a, k) * Di[lane][k];
            if (lane < jb) L[(long)i * n + j0 + lane] = (S)out;
        }
        __syncthreads();
        // (3) trailing update of the lower triangle, one 32 x 32 tile per warp
        const int R = P - p - 1;
        const int ntile = R * (R + 1) / 2;
        WarpTiles<C>& W = wt[warp];
        for (int t = warp; t < ntile; t += NW) {
            int ii = 0;
            while ((ii + 1) * (ii + 2) / 2 <= t) ++ii;
            const int kk = t - ii * (ii + 1) / 2;
            const int I0 = (p + 1 + ii) * 32, K0 = (p + 1 + kk) * 32;
            {
                // Ks[k][j] = L[K0+j][j0+k] (lane j reads its row), Is[i][k] = L[I0+i][j0+k]
                C kv[32], iv[32];
                const bool kr = (K0 + lane < n);
#pragma unroll
                for (int k = 0; k < 32; ++k) kv[k] = (kr && k < jb) ? (C)L[(long)(K0 + lane) * n + j0 + k] : C(0);
#pragma unroll
                for (int r = 0; r < 32; ++r)
                    iv[r] = (I0 + r < n && lane < jb) ? (C)L[(long)(I0 + r) * n + j0 + lane] : C(0);
#pragma unroll
                for (int k = 0; k < 32; ++k) W.Ks[k][lane] = kv[k];
#pragma unroll
                for (int r = 0; r < 32; ++r) W.Is[r][lane] = iv[r];
            }
            __syncwarp();
            C acc[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[j] = C(0);
#pragma unroll 2
            for (int k = 0; k < 32; ++k) {
                const C a = W.Is[lane][k];
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[j] = fma(a, W.Ks[k][j], acc[j]);
            }
            const int row = I0 + lane;
            if (row < n) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int col = K0 + j;
                    if (col < n && (ii != kk || j <= lane)) {
                        const long e = (long)row * n + col;
                        L[e] = (S)((C)L[e] - acc[j]);
                    }
                }
            }
            __syncwarp();
        }
        __syncthreads();
    }
    // inverse: T_IJ = -T_II sum_{K=J}^{I-1} L_IK T_KJ, block rows in order
    for (int I = 1; I < P; ++I) {
        const int I0 = I * 32;
        WarpTiles<C>& W = wt[warp];
        for (int J = warp; J < I; J += NW) {
            const int J0 = J * 32;
            C acc[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[j] = C(0);
            for (int K = J; K < I; ++K) {
                const int K0 = K * 32;
                // Ks[k][j] = T[K0+k][J0+j]; Is[i][k] = L[I0+i][K0+k]
                {
                    C kv[32], iv[32];
#pragma unroll
                    for (int r = 0; r < 32; ++r) {
                        kv[r] = (K0 + r < n && J0 + lane < n) ? (C)Tm[(long)(K0 + r) * n + J0 + lane] : C(0);
                        iv[r] = (I0 + r < n && K0 + lane < n) ? (C)L[(long)(I0 + r) * n + K0 + lane] : C(0);
                    }
#pragma unroll
                    for (int r = 0; r < 32; ++r) {
                        W.Ks[r][lane] = kv[r];
                        W.Is[r][lane] = iv[r];
                    }
                }
                __syncwarp();
#pragma unroll 2
                for (int k = 0; k < 32; ++k) {
                    const C a = W.Is[lane][k];
#pragma unroll
                    for (int j = 0; j < 32; ++j) acc[j] = fma(a, W.Ks[k][j], acc[j]);
                }
                __syncwarp();
            }
            // T_IJ = -T_II S: stage S rows in Ks, T_II rows in Is
            for (int j = 0; j < 32; ++j) W.Ks[lane][j] = acc[j];
            for (int r = 0; r < 32; ++r)
                W.Is[r][lane] = (I0 + r < n && I0 + lane < n) ? (C)Tm[(long)(I0 + r) * n + I0 + lane] : C(0);
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[j] = C(0);
#pragma unroll 4
            for (int m = 0; m < 32; ++m) {
                const C a = W.Is[lane][m];
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[j] = fma(a, W.Ks[m][j], acc[j]);
            }
            const int row = I0 + lane;
            if (row < n) {
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (J0 + j < n) Tm[(long)row * n + J0 + j] = (S)(-acc[j]);
            }
            __syncwarp();
        }
        __syncthreads();
    }
    if (tid == 0) {
        st->ndrop = s_ndrop;
        st->nonfinite = s_nonfinite;
        st->min_ratio = s_minratio > 1e299 ? 0.0 : s_minratio;
        st->trace = tr;
        st->max_diag = mx;
    }
}

}  // namespace

template <class S, class C>
void chol_inv(Ctx& c, int n, const S* G, S* L, S* T, double shift_rel, double drop_rel, CholStatus* st) {
    if (n <= 0) return;
    constexpr int NT = sizeof(C) == 8 ? 256 : 512;
    const size_t smem = (NT / 32) * sizeof(WarpTiles<C>);
    static bool attr = false;
    if (!attr) {
        TT_CUDA(cudaFuncSetAttribute(chol_inv_kernel<S, C, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        attr = true;
    }
    ProfScope ps(c, "chol_inv", 2.0 * (double)n * n * n / 3.0, 3.0 * sizeof(S) * n * n);
    chol_inv_kernel<S, C, NT><<<1, NT, smem, c.stream>>>(n, G, L, T, shift_rel, drop_rel, st);
    TT_LAUNCHED(c);
}

template void chol_inv<double, double>(Ctx&, int, const double*, double*, double*, double, double, CholStatus*);
template void chol_inv<float, float>(Ctx&, int, const float*, float*, float*, double, double, CholStatus*);

}  // namespace ttgb
