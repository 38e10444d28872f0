// Blocked Cholesky factorization with rank drop and explicit inverse of the
// factor, one CTA, for the small r x r Gram matrices of the Cholesky QR
// passes of TT-round:  G + s I = L L^T, T = L^{-1}.
//
// Right-looking over 32-column panels p.  Per panel, three phases separated
// by block barriers:
//  1. warp 0 factors the 32 x 32 diagonal block (each lane holds one row in
//     registers, columns are eliminated with warp shuffles; a pivot below the
//     drop threshold zeroes its column) and inverts it (each lane holds one
//     column of the inverse);
//  2. all warps solve the panel rows below (L_ip = A_ip L_pp^{-T}) and
//     finalize block row p of the inverse, T_pJ = -T_pp W_pJ (J < p);
//  3. all warps apply the rank-32 updates, one 32 x 32 tile per warp at a
//     time: the trailing lower triangle A_IK -= L_Ip L_Kp^T (p < K <= I) and
//     the inverse accumulators W_IJ += L_Ip T_pJ (I > p, J <= p), kept in the
//     lower blocks of T until their row is finalized.
// This is block forward substitution for L T = I run right-looking, so the
// inverse needs no phase of its own.  The matrices live in global memory
// (L2-resident at these sizes); each warp stages its tiles in its own
// shared-memory slots.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "internal.h"

namespace ttgb {

namespace {

constexpr unsigned FULL = 0xffffffffu;

template <class C>
struct WarpTiles {
    C Ks[32][32];  // read by broadcast: Ks[k][j]
    C Is[32][33];  // read one row per lane: Is[i][k]
};

// acc[j] = sum_k Is[lane][k] * Ks[k][j]
template <class C>
__device__ __forceinline__ void tile_mac(const WarpTiles<C>& W, int lane, C (&acc)[32]) {
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = C(0);
#pragma unroll 2
    for (int k = 0; k < 32; ++k) {
        const C a = W.Is[lane][k];
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = fma(a, W.Ks[k][j], acc[j]);
    }
}

template <class S, class C, int NT>
__global__ void __launch_bounds__(NT)
chol_inv_kernel(int n, const S* __restrict__ G, S* __restrict__ L, S* __restrict__ Tm, double shift_rel,
                double drop_rel, CholStatus* st) {
    extern __shared__ __align__(16) unsigned char ci_smem[];
    constexpr int NW = NT / 32;
    WarpTiles<C>* wt = reinterpret_cast<WarpTiles<C>*>(ci_smem);
    __shared__ C Ds[32][33];  // L_pp
    __shared__ C Di[32][33];  // L_pp^{-1}
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
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tr += __shfl_xor_sync(FULL, tr, o);
        mx = fmax(mx, __shfl_xor_sync(FULL, mx, o));
    }
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
    WarpTiles<C>& W = wt[warp];
    for (int p = 0; p < P; ++p) {
        const int j0 = p * 32, jb = min(32, n - j0);
        // ---- 1. diagonal block, warp 0: factor (rows in registers) and invert
        if (warp == 0) {
            C d[32];
#pragma unroll
            for (int k = 0; k < 32; ++k)
                d[k] = (lane < jb && k <= lane) ? (C)L[(long)(j0 + lane) * n + j0 + k] : C(0);
            const double gd = (lane < jb) ? (double)G[(long)(j0 + lane) * n + j0 + lane] + shift : 1.0;
            int ndrop = 0, nonfin = 0;
            double minr = 1e300;
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                if (c < jb) {
                    const C piv = __shfl_sync(FULL, d[c], c);
                    const double orig = __shfl_sync(FULL, gd, c);
                    const bool fin = isfinite((double)piv);
                    const bool keep = fin && (double)piv > tau && piv > C(0);
                    const C dc = keep ? sqrt(piv) : C(0);
                    const C inv = keep ? C(1) / dc : C(0);
                    if (lane == c) d[c] = dc;
                    else if (lane > c) d[c] *= inv;
#pragma unroll
                    for (int k = c + 1; k < 32; ++k) {
                        const C lkc = __shfl_sync(FULL, d[c], k);
                        if (lane >= k) d[k] = fma(-d[c], lkc, d[k]);
                    }
                    nonfin |= !fin;
                    if (keep) minr = fmin(minr, orig > 0.0 ? (double)piv / orig : 0.0);
                    else ++ndrop;
                }
            }
#pragma unroll
            for (int k = 0; k < 32; ++k) Ds[lane][k] = (k <= lane) ? d[k] : C(0);
            __syncwarp();
            // column `lane` of L_pp^{-1} by forward substitution, in registers
            C x[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const C lii = Ds[i][i];
                C s = (i == lane) ? C(1) : C(0);
#pragma unroll
                for (int k = 0; k < i; ++k) s = fma(-Ds[i][k], x[k], s);
                x[i] = (lii != C(0) && i < jb) ? s / lii : C(0);
            }
#pragma unroll
            for (int i = 0; i < 32; ++i) Di[i][lane] = x[i];
            __syncwarp();
            if (lane < jb) {
                for (int k = 0; k <= lane; ++k) {
                    L[(long)(j0 + lane) * n + j0 + k] = (S)Ds[lane][k];
                    Tm[(long)(j0 + lane) * n + j0 + k] = (S)Di[lane][k];
                }
            }
            if (lane == 0) {
                s_ndrop += ndrop;
                s_nonfinite |= nonfin;
                s_minratio = fmin(s_minratio, minr);
            }
        }
        __syncthreads();
        // ---- 2a. panel rows below: L[i, panel] = A[i, panel] L_pp^{-T}
        for (int i = j0 + jb + warp; i < n; i += NW) {
            const C a = (lane < jb) ? (C)L[(long)i * n + j0 + lane] : C(0);
            C out = C(0);
#pragma unroll
            for (int k = 0; k < 32; ++k) out = fma(__shfl_sync(FULL, a, k), Di[lane][k], out);
            if (lane < jb) L[(long)i * n + j0 + lane] = (S)out;
        }
        // ---- 2b. block row p of the inverse: T_pJ = -T_pp W_pJ, J < p
        for (int J = warp; J < p; J += NW) {
            const int J0 = J * 32;
            {
                C kv[32];
#pragma unroll
                for (int m = 0; m < 32; ++m)
                    kv[m] = (j0 + m < n) ? (C)Tm[(long)(j0 + m) * n + J0 + lane] : C(0);
#pragma unroll
                for (int m = 0; m < 32; ++m) {
                    W.Ks[m][lane] = kv[m];
                    W.Is[m][lane] = Di[m][lane];
                }
            }
            __syncwarp();
            C acc[32];
            tile_mac(W, lane, acc);
            if (lane < jb) {
#pragma unroll
                for (int j = 0; j < 32; ++j) Tm[(long)(j0 + lane) * n + J0 + j] = (S)(-acc[j]);
            }
            __syncwarp();
        }
        __syncthreads();
        // ---- 3. rank-32 updates: trailing lower triangle and inverse accumulators
        const int R = P - p - 1;
        const int n_syrk = R * (R + 1) / 2;
        const int n_w = R * (p + 1);
        for (int t = warp; t < n_syrk + n_w; t += NW) {
            int I0, K0 = 0, J0 = 0;
            bool syrk = t < n_syrk;
            bool diag_tile = false;
            if (syrk) {
                int ii = 0;
                while ((ii + 1) * (ii + 2) / 2 <= t) ++ii;
                const int kk = t - ii * (ii + 1) / 2;
                I0 = (p + 1 + ii) * 32;
                K0 = (p + 1 + kk) * 32;
                diag_tile = (ii == kk);
            } else {
                const int u = t - n_syrk;
                I0 = (p + 1 + u / (p + 1)) * 32;
                J0 = (u % (p + 1)) * 32;
            }
            {
                C kv[32], iv[32];
                if (syrk) {
                    // Ks[c][j] = L[K0+j][j0+c]: lane j reads its row
                    const bool kr = (K0 + lane < n);
#pragma unroll
                    for (int c = 0; c < 32; ++c) kv[c] = (kr && c < jb) ? (C)L[(long)(K0 + lane) * n + j0 + c] : C(0);
                } else {
                    // Ks[c][j] = T[j0+c][J0+j]
#pragma unroll
                    for (int c = 0; c < 32; ++c) kv[c] = (j0 + c < n) ? (C)Tm[(long)(j0 + c) * n + J0 + lane] : C(0);
                }
#pragma unroll
                for (int r = 0; r < 32; ++r)
                    iv[r] = (I0 + r < n && lane < jb) ? (C)L[(long)(I0 + r) * n + j0 + lane] : C(0);
#pragma unroll
                for (int c = 0; c < 32; ++c) W.Ks[c][lane] = kv[c];
#pragma unroll
                for (int r = 0; r < 32; ++r) W.Is[r][lane] = iv[r];
            }
            __syncwarp();
            C acc[32];
            tile_mac(W, lane, acc);
            const int row = I0 + lane;
            if (row < n) {
                if (syrk) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int col = K0 + j;
                        if (col < n && (!diag_tile || j <= lane)) {
                            const long e = (long)row * n + col;
                            L[e] = (S)((C)L[e] - acc[j]);
                        }
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int col = J0 + j;
                        if (col < n) {
                            const long e = (long)row * n + col;
                            Tm[e] = (S)((C)Tm[e] + acc[j]);
                        }
                    }
                }
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
    // panel in shared memory when it fits (n <= 512 FP32, n <= 256 FP64)
    if (chol_inv_smem<S, C>(c, n, G, L, T, shift_rel, drop_rel, st)) return;
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
