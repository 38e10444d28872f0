// Cholesky factorization with rank drop and explicit inverse of the factor,
// one CTA, with the working panel held in shared memory (n <= 512 in FP32,
// n <= 256 in FP64):  G + s I = L L^T,  T = L^{-1}.
//
// Same right-looking scheme as chol_inv.cu (32-column panels; the inverse
// accumulated as W_IJ += L_Ip T_pJ and finalized as T_pJ = -T_pp W_pJ), with
// three changes that remove the latency the global-memory version waits on:
//  - the current panel L[:, p] is kept in shared memory in both orientations
//    (row-major for the per-lane row reads, transposed for the broadcast
//    column reads), and so is block row p of T, so a tile update reads its
//    operands from shared memory and only its 32 x 32 output goes to L2,
//    loaded before the arithmetic so the load latency overlaps it;
//  - the 32 x 32 diagonal block is factored by the whole CTA (a single warp
//    doing it serially was the critical path), with reciprocal pivots;
//  - the panel solve keeps four rows in flight per warp.
#include <cuda_runtime.h>
#include <math.h>

#include "internal.h"

namespace ttgb {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// factor + invert the diagonal block p with the whole CTA: column by column,
// thread 0 takes the pivot decision, the column below it is scaled and the
// trailing triangle of the block updated in parallel (two barriers per
// column); then warp 0 forms the inverse (lane j = column j, in registers,
// multiplying by the reciprocal pivots).  Writes Ds, Di and the diagonal
// blocks of L and T in global memory.
template <class S, class C, int NT>
__device__ void factor_diag_cta(int n, int p, const S* __restrict__ G, S* __restrict__ L, S* __restrict__ Tm,
                                double shift, double tau, C (*Ds)[33], C (*Di)[33], C* s_inv, int* s_ndrop,
                                int* s_nonfin, double* s_minratio) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int j0 = p * 32, jb = min(32, n - j0);
    for (int e = tid; e < 32 * 32; e += NT) {
        const int r = e >> 5, k = e & 31;
        Ds[r][k] = (r < jb && k <= r) ? (C)L[(long)(j0 + r) * n + j0 + k] : C(0);
    }
    // original diagonal (for the pivot ratio), loaded once, off the column chain
    if (tid < jb) Di[tid][0] = (C)((double)G[(long)(j0 + tid) * n + j0 + tid] + shift);
    __syncthreads();
    const C tau_c = (C)tau;
    for (int c = 0; c < jb; ++c) {
        if (tid == 0) {
            const C piv = Ds[c][c];
            const C orig = Di[c][0];
            const bool fin = isfinite(piv);
            const bool keep = fin && piv > tau_c && piv > C(0);
            const C dc = keep ? sqrt(piv) : C(0);
            const C inv = keep ? C(1) / dc : C(0);
            Ds[c][c] = dc;
            s_inv[c] = inv;
            if (!fin) *s_nonfin = 1;
            if (keep) *s_minratio = fmin(*s_minratio, orig > C(0) ? (double)(piv / orig) : 0.0);
            else *s_ndrop += 1;
        }
        __syncthreads();
        // trailing update of the block with the unscaled column c: A_rk -= a_rc a_kc / piv
        const C inv = s_inv[c];
        const C inv2 = inv * inv;
        for (int e = tid; e < 32 * 32; e += NT) {
            const int r = e >> 5, k = e & 31;
            if (k > c && k <= r && r < jb) Ds[r][k] = fma(-Ds[r][c] * inv2, Ds[k][c], Ds[r][k]);
        }
        __syncthreads();
        if (tid > c && tid < jb) Ds[tid][c] *= inv;  // scale column c (read again only after the next barrier)
    }
    __syncthreads();
    if (warp == 0) {
        C x[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            C sacc = (i == lane) ? C(1) : C(0);
#pragma unroll
            for (int k = 0; k < i; ++k) sacc = fma(-Ds[i][k], x[k], sacc);
            x[i] = (i < jb) ? sacc * s_inv[i] : C(0);
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) Di[i][lane] = x[i];
    }
    __syncthreads();
    for (int e = tid; e < 32 * 32; e += NT) {
        const int r = e >> 5, k = e & 31;
        if (r < jb && k <= r) {
            L[(long)(j0 + r) * n + j0 + k] = (S)Ds[r][k];
            Tm[(long)(j0 + r) * n + j0 + k] = (S)Di[r][k];
        }
    }
}

// 16-byte vector of the compute type, and acc[0..W) += a * v
template <class C>
struct Vec16;
template <>
struct Vec16<float> {
    using T = float4;
    static constexpr int W = 4;
    __device__ __forceinline__ static void fma(float a, const float4 v, float* acc) {
        acc[0] = fmaf(a, v.x, acc[0]);
        acc[1] = fmaf(a, v.y, acc[1]);
        acc[2] = fmaf(a, v.z, acc[2]);
        acc[3] = fmaf(a, v.w, acc[3]);
    }
};
template <>
struct Vec16<double> {
    using T = double2;
    static constexpr int W = 2;
    __device__ __forceinline__ static void fma(double a, const double2 v, double* acc) {
        acc[0] = ::fma(a, v.x, acc[0]);
        acc[1] = ::fma(a, v.y, acc[1]);
    }
};

// one 32 x 32 tile of the rank-32 update of panel p (task t)
template <class S, class C>
__device__ void update_tile(int n, int npad, int p, int t, int nsy, S* __restrict__ L, S* __restrict__ Tm,
                            const C* __restrict__ Pn, const C* __restrict__ PT, const C* __restrict__ TR) {
    const int lane = threadIdx.x & 31;
    int I0, C0;
    bool syrk = t < nsy, diag_tile = false;
    if (syrk) {
        int ii = 0;
        while ((ii + 1) * (ii + 2) / 2 <= t) ++ii;
        const int kk = t - ii * (ii + 1) / 2;
        I0 = (p + 1 + ii) * 32;
        C0 = (p + 1 + kk) * 32;
        diag_tile = (ii == kk);
    } else {
        const int u = t - nsy;
        I0 = (p + 1 + u / (p + 1)) * 32;
        C0 = (u % (p + 1)) * 32;
    }
    const int row = I0 + lane;
    S* out = syrk ? L : Tm;
    // prefetch this lane's 32 outputs
    C o[32];
    const bool rv = row < n;
#pragma unroll
    for (int j = 0; j < 32; ++j) o[j] = (rv && C0 + j < n) ? (C)out[(long)row * n + C0 + j] : C(0);
    C acc[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = C(0);
    const C* rowp = Pn + (long)row * 33;
    const C* colp = (syrk ? PT : TR) + C0;
    // the broadcast row colp[c * npad + 0..31] is 16-byte aligned (C0 and npad
    // are multiples of 32): read it with 16-byte loads
    using V = typename Vec16<C>::T;
    constexpr int W = Vec16<C>::W;
#pragma unroll 2
    for (int c = 0; c < 32; ++c) {
        const C a = rowp[c];
        const V* b = reinterpret_cast<const V*>(colp + (long)c * npad);
#pragma unroll
        for (int j = 0; j < 32 / W; ++j) Vec16<C>::fma(a, b[j], acc + j * W);
    }
    if (rv) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int col = C0 + j;
            if (col < n) {
                if (syrk) {
                    if (!diag_tile || j <= lane) out[(long)row * n + col] = (S)(o[j] - acc[j]);
                } else {
                    out[(long)row * n + col] = (S)(o[j] + acc[j]);
                }
            }
        }
    }
}

template <class S, class C, int NT>
__global__ void __launch_bounds__(NT)
chol_inv_smem_kernel(int n, int npad, const S* __restrict__ G, S* __restrict__ L, S* __restrict__ Tm,
                     double shift_rel, double drop_rel, CholStatus* st) {
    extern __shared__ __align__(16) unsigned char cs_smem[];
    constexpr int NW = NT / 32;
    C* Pn = reinterpret_cast<C*>(cs_smem);  // [npad][33]
    C* PT = Pn + (long)npad * 33;            // [32][npad]
    C* TR = PT + 32L * npad;                 // [32][npad]
    __shared__ C Ds[32][33];
    __shared__ C Di[32][33];
    __shared__ C s_inv[32];
    __shared__ double shd[32];
    __shared__ int s_ndrop, s_nonfinite;
    __shared__ double s_minratio;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

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

    const long smem_elems = (long)npad * 33 + 64L * npad;
    for (long e = tid; e < smem_elems; e += NT) Pn[e] = C(0);
    for (int i = warp; i < n; i += NW) {
        for (int k = lane; k < n; k += 32) {
            const long e = (long)i * n + k;
            L[e] = (k <= i) ? (S)((C)G[e] + (i == k ? (C)shift : C(0))) : S(0);
            Tm[e] = S(0);
        }
    }
    __syncthreads();

    const int P = (n + 31) / 32;
    for (int p = 0; p < P; ++p) {
        const int j0 = p * 32, jb = min(32, n - j0);
        // ---- phase 1: diagonal block, whole CTA
        factor_diag_cta<S, C, NT>(n, p, G, L, Tm, shift, tau, Ds, Di, s_inv, &s_ndrop, &s_nonfinite, &s_minratio);
        // ---- phase 2a: diagonal block into the shared panel copies
        for (int r = warp; r < 32; r += NW) {
            const int i = j0 + r;
            const C v = (r < jb && lane < jb && lane <= r) ? Ds[r][lane] : C(0);
            Pn[(long)i * 33 + lane] = v;
            PT[(long)lane * npad + i] = v;
            TR[(long)r * npad + j0 + lane] = (r < jb && lane < jb) ? Di[r][lane] : C(0);
        }
        // ---- phase 2b: panel rows below, four in flight per warp
        for (int i0 = j0 + jb + warp; i0 < n; i0 += 4 * NW) {
            C a[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = i0 + q * NW;
                a[q] = (i < n && lane < jb) ? (C)L[(long)i * n + j0 + lane] : C(0);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = i0 + q * NW;
                C out = C(0);
#pragma unroll
                for (int k = 0; k < 32; ++k) out = fma(__shfl_sync(FULL, a[q], k), Di[lane][k], out);
                if (i < n) {
                    const C v = (lane < jb) ? out : C(0);
                    if (lane < jb) L[(long)i * n + j0 + lane] = (S)out;
                    Pn[(long)i * 33 + lane] = v;
                    PT[(long)lane * npad + i] = v;
                }
            }
        }
        // ---- phase 2c: block row p of the inverse, T_pJ = -T_pp W_pJ (J < p)
        for (int J = warp; J < p; J += NW) {
            const int J0 = J * 32;
            // stage W_pJ in TR (block row p, columns J0..J0+31)
#pragma unroll 4
            for (int m = 0; m < 32; ++m)
                TR[(long)m * npad + J0 + lane] = (m < jb) ? (C)Tm[(long)(j0 + m) * n + J0 + lane] : C(0);
            __syncwarp();
            C acc[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[j] = C(0);
#pragma unroll 2
            for (int m = 0; m < 32; ++m) {
                const C a = Di[lane][m];
                const C* b = TR + (long)m * npad + J0;
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[j] = fma(a, b[j], acc[j]);
            }
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                TR[(long)lane * npad + J0 + j] = -acc[j];
                if (lane < jb) Tm[(long)(j0 + lane) * n + J0 + j] = (S)(-acc[j]);
            }
            __syncwarp();
        }
        __syncthreads();
        // ---- phase 3: rank-32 updates, one tile per warp at a time
        const int R = P - p - 1;
        if (R > 0) {
            const int nsy = R * (R + 1) / 2;
            const int ntask = nsy + R * (p + 1);
            for (int t = warp; t < ntask; t += NW) update_tile<S, C>(n, npad, p, t, nsy, L, Tm, Pn, PT, TR);
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
bool chol_inv_smem(Ctx& c, int n, const S* G, S* L, S* T, double shift_rel, double drop_rel, CholStatus* st) {
    constexpr int NT = sizeof(C) == 8 ? 256 : 512;
    constexpr int NMAX = sizeof(C) == 8 ? 256 : 512;
    if (n <= 0 || n > NMAX) return false;
    const int npad = ((n + 31) / 32) * 32;
    const size_t smem = sizeof(C) * ((size_t)npad * 33 + 64 * (size_t)npad);
    const size_t smem_max = sizeof(C) * ((size_t)NMAX * 33 + 64 * (size_t)NMAX);
    static bool attr = false;
    if (!attr) {
        TT_CUDA(cudaFuncSetAttribute(chol_inv_smem_kernel<S, C, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem_max));
        attr = true;
    }
    ProfScope ps(c, "chol_inv", 2.0 * (double)n * n * n / 3.0, 3.0 * sizeof(S) * n * n);
    chol_inv_smem_kernel<S, C, NT><<<1, NT, smem, c.stream>>>(n, npad, G, L, T, shift_rel, drop_rel, st);
    TT_LAUNCHED(c);
    return true;
}

template bool chol_inv_smem<double, double>(Ctx&, int, const double*, double*, double*, double, double, CholStatus*);
template bool chol_inv_smem<float, float>(Ctx&, int, const float*, float*, float*, double, double, CholStatus*);

}  // namespace ttgb
