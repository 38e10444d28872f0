// CUDA-core kernels of the TT library: tiled GEMM / split-K Gram, small
// dense factorizations (Cholesky with rank drop, triangular inverse, one-sided
// Jacobi SVD), reductions and the block scatter of the TT sum.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "internal.h"

namespace ttgb {

// ------------------------------------------------------------------ GEMM
// 64x64 output tile, BK = 16, 256 threads, 4x4 outputs per thread (strided
// by 16 so that shared-memory reads broadcast).  MODE 0: plain (blockIdx.z
// = batch).  MODE 1: Gram, only tiles with tile_row >= tile_col, blockIdx.z
// = split of K, result atomically added into C of type CT.  MODE 2: split-K
// of a plain product (few output tiles, long K: the contractions of a TT dot
// against a low-rank tensor), alpha times each partial added atomically into
// a zeroed C.
namespace {

constexpr int GBM = 64, GBN = 64, GBK = 16;

template <class T, class CT, bool TA, bool TB, int MODE>
__global__ void __launch_bounds__(256)
gemm_kernel(int M, int N, long K, T alpha, const T* __restrict__ A, long lda,
            const T* __restrict__ B, long ldb, T beta, CT* __restrict__ C, long ldc, long sA,
            long sB, long sC, long kchunk, int tri) {
    __shared__ T As[GBK][GBM + 1];
    __shared__ T Bs[GBK][GBN + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    long kbeg = 0, kend = K;
    if (MODE == 0) {
        A += blockIdx.z * sA;
        B += blockIdx.z * sB;
        C += blockIdx.z * sC;
    } else {
        if (MODE == 1 && blockIdx.x > blockIdx.y) return;  // upper tiles of a symmetric result
        kbeg = (long)blockIdx.z * kchunk;
        kend = min(K, kbeg + kchunk);
        if (kbeg >= kend) return;
    }
    if (MODE != 1 && tri_skip_tile(tri, m0, n0, GBM)) return;
    if (MODE != 1) tri_krange(tri, m0, n0, GBM, GBN, kbeg, kend);  // tile multiples of GBK
    if (MODE == 2 && kbeg >= kend) return;  // a zero partial: nothing to add
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

    for (long k0 = kbeg; k0 < kend; k0 += GBK) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int e = tid + l * 256;
            int mm, kk;
            if (!TA) { kk = e & 15; mm = e >> 4; } else { mm = e & 63; kk = e >> 6; }
            const long gm = m0 + mm, gk = k0 + kk;
            T v = T(0);
            if (gm < M && gk < kend) v = TA ? A[gk * lda + gm] : A[gm * lda + gk];
            As[kk][mm] = v;
        }
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int e = tid + l * 256;
            int nn, kk;
            if (!TB) { nn = e & 63; kk = e >> 6; } else { kk = e & 15; nn = e >> 4; }
            const long gn = n0 + nn, gk = k0 + kk;
            T v = T(0);
            if (gn < N && gk < kend) v = TB ? B[gn * ldb + gk] : B[gk * ldb + gn];
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const long gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long gn = n0 + tx + 16 * j;
            if (gn >= N) continue;
            if (MODE != 1 && (tri & TRI_C_LOWER) && gn > gm) continue;  // lower triangle only
            if (MODE == 0) {
                T v = alpha * acc[i][j];
                if (beta != T(0)) v += beta * (T)C[gm * ldc + gn];
                C[gm * ldc + gn] = (CT)v;
            } else if (MODE == 1) {
                atomicAdd(&C[gm * ldc + gn], (CT)acc[i][j]);
            } else {
                atomicAdd(&C[gm * ldc + gn], (CT)(alpha * acc[i][j]));
            }
        }
    }
}

// Products of r x r size (the series pass, the factor products, the blocked
// Cholesky's panel and trailing products): 32 x 32 output tile per CTA (169
// CTAs at r = 400), 256 threads in 4 groups that split each K chunk, 4 x 4
// outputs per thread read as 16-byte vectors from k-major shared tiles, the
// groups' partial tiles summed through shared memory at the end.  A chunk
// (KC of K) of both operands is staged by element-wise asynchronous copies
// (zero-filled outside the matrices, any layout or alignment).  No split
// over CTAs, no atomics.
constexpr int RT = 32;

template <class T>
struct Vec4;
template <>
struct Vec4<float> {
    __device__ __forceinline__ static void ld(const float* p, float* x) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    }
};
template <>
struct Vec4<double> {
    __device__ __forceinline__ static void ld(const double* p, double* x) {
        const double2 u = *reinterpret_cast<const double2*>(p), v = *reinterpret_cast<const double2*>(p + 2);
        x[0] = u.x; x[1] = u.y; x[2] = v.x; x[3] = v.y;
    }
};

template <class T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src, bool ok) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "n"(sizeof(T)), "r"(ok ? (int)sizeof(T) : 0));
}

template <class T, bool TA, bool TB>
__global__ void __launch_bounds__(256)
rgemm_kernel(int M, int N, long K, T alpha, const T* __restrict__ A, long lda, const T* __restrict__ B, long ldb,
             T beta, T* __restrict__ C, long ldc, int tri) {
    constexpr int KC = sizeof(T) == 4 ? 128 : 64;
    constexpr int LDK = RT + 4;            // k-major rows of 32 (+ pad), 16-byte aligned
    constexpr int PER = RT * KC / 256;     // staged elements per thread and operand
    constexpr int SM = 2 * KC * LDK > 3 * RT * (RT + 1) ? 2 * KC * LDK : 3 * RT * (RT + 1);
    __shared__ __align__(16) T smem[SM];
    T* As = smem;             // As[k][i] = op(A)(m0 + i, k0 + k)
    T* Bs = smem + KC * LDK;  // Bs[k][j] = op(B)(k0 + k, n0 + j)
    const int tid = threadIdx.x;
    const int grp = tid >> 6, t = tid & 63, ti = t >> 3, tj = t & 7;
    const int m0 = blockIdx.y * RT, n0 = blockIdx.x * RT;
    if (tri_skip_tile(tri, m0, n0, RT)) return;
    long kb = 0, ke = K;
    tri_krange(tri, m0, n0, RT, RT, kb, ke);
    T acc[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = T(0);
    for (long k0 = kb; k0 < ke; k0 += KC) {
        const int kc = (int)min((long)KC, ke - k0);
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            // element e of the chunk, the global operand's contiguous index fastest
            const int e = tid + 256 * q;
            {
                const int k = TA ? e / RT : e % KC, i = TA ? e % RT : e / KC;
                const long gm = m0 + i;
                const bool ok = gm < M && k < kc;
                cp_async_elem(As + k * LDK + i, ok ? (TA ? A + (k0 + k) * lda + gm : A + gm * lda + k0 + k) : A, ok);
            }
            {
                const int k = TB ? e % KC : e / RT, j = TB ? e / KC : e % RT;
                const long gn = n0 + j;
                const bool ok = gn < N && k < kc;
                cp_async_elem(Bs + k * LDK + j, ok ? (TB ? B + gn * ldb + k0 + k : B + (k0 + k) * ldb + gn) : B, ok);
            }
        }
        asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
#pragma unroll 4
        for (int k = grp; k < kc; k += 4) {
            T a[4], b[4];
            Vec4<T>::ld(As + k * LDK + 4 * ti, a);
            Vec4<T>::ld(Bs + k * LDK + 4 * tj, b);
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
        }
        __syncthreads();
    }
    // groups 1..3 leave their partial tiles in shared memory, group 0 sums
    T* red = smem;  // [3][RT][RT + 1]
    if (grp > 0) {
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) red[((grp - 1) * RT + 4 * ti + x) * (RT + 1) + 4 * tj + y] = acc[x][y];
    }
    __syncthreads();
    if (grp == 0) {
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const long gm = m0 + 4 * ti + x;
#pragma unroll
            for (int y = 0; y < 4; ++y) {
                const long gn = n0 + 4 * tj + y;
                T v = acc[x][y];
#pragma unroll
                for (int h = 0; h < 3; ++h) v += red[(h * RT + 4 * ti + x) * (RT + 1) + 4 * tj + y];
                if (gm < M && gn < N && !((tri & TRI_C_LOWER) && gn > gm)) {
                    v = alpha * v;
                    if (beta != T(0)) v += beta * C[gm * ldc + gn];
                    C[gm * ldc + gn] = v;
                }
            }
        }
    }
}

template <class T, class CT, int MODE>
void launch_gemm(Ctx& c, bool tA, bool tB, dim3 grid, int M, int N, long K, T alpha,
                 const T* A, long lda, const T* B, long ldb, T beta, CT* C, long ldc, long sA,
                 long sB, long sC, long kchunk, int tri) {
#define TT_GEMM_CASE(TA_, TB_)                                                            \
    gemm_kernel<T, CT, TA_, TB_, MODE><<<grid, 256, 0, c.stream>>>(                      \
        M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sA, sB, sC, kchunk, tri)
    if (!tA && !tB) TT_GEMM_CASE(false, false);
    else if (!tA && tB) TT_GEMM_CASE(false, true);
    else if (tA && !tB) TT_GEMM_CASE(true, false);
    else TT_GEMM_CASE(true, true);
#undef TT_GEMM_CASE
    TT_LAUNCHED(c);
}

}  // namespace

double gemm_flops(long M, long N, long K, int tri) {
    // sum_{i < rows} of the k-range length min(K, i + 1) (lower) or
    // max(0, K - i) (upper)
    auto lower_pairs = [](long rows, long K) {
        const long t = std::min(rows, K);
        return (double)t * (t + 1) / 2.0 + (double)(rows - t) * K;
    };
    auto upper_pairs = [](long rows, long K) {
        const long t = std::min(rows, K);
        return (double)t * K - (double)t * (t - 1) / 2.0;
    };
    double f = 2.0 * M * N * (double)K;
    if (tri & TRI_A_LOWER) f = std::min(f, 2.0 * N * lower_pairs(M, K));
    if (tri & TRI_A_UPPER) f = std::min(f, 2.0 * N * upper_pairs(M, K));
    if (tri & TRI_B_UPPER) f = std::min(f, 2.0 * M * lower_pairs(N, K));
    if (tri & TRI_B_LOWER) f = std::min(f, 2.0 * M * upper_pairs(N, K));
    if (tri & TRI_C_LOWER) f = std::min(f, 2.0 * K * lower_pairs(M, N));
    return f;
}

template <class T>
void gemm(Ctx& c, bool tA, bool tB, int M, int N, int K, T alpha, const T* A, long lda,
          const T* B, long ldb, T beta, T* C, long ldc, int batch, long sA, long sB, long sC, int tri) {
    if (M <= 0 || N <= 0 || batch <= 0) return;
    if (K <= 0) {
        // C = beta C: degenerate product
        if (beta == T(0)) {
            for (int z = 0; z < batch; ++z)
                TT_CUDA(cudaMemset2DAsync(C + z * sC, ldc * sizeof(T), 0, N * sizeof(T), M, c.stream));
            return;
        }
        throw_status(TT_ERR_ARG, "gemm with K = 0 and beta != 0");
    }
    if (batch > 65535) throw_status(TT_ERR_ARG, "gemm batch too large");
    if constexpr (sizeof(T) == 4) {
        // the 128 x 128 kernel when it fills at least half the SMs; smaller
        // products (the r x r ones) take 64 x 64 tiles, split over K below
        const long tiles128 = (long)((N + 127) / 128) * ((M + 127) / 128) * batch;
        if (2 * tiles128 >= c.sm_count &&
            sgemm(c, tA, tB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, batch, sA, sB, sC, tri))
            return;
    }
    if (batch == 1 && K <= 2048 && (long)((M + RT - 1) / RT) * ((N + RT - 1) / RT) <= 2L * c.sm_count) {
        ProfScope ps(c, sizeof(T) == 8 ? "rgemm_f64" : "rgemm_f32", gemm_flops(M, N, K, tri),
                     sizeof(T) * ((double)M * K + (double)K * N + 2.0 * M * N));
        dim3 g((N + RT - 1) / RT, (M + RT - 1) / RT);
#define TT_RGEMM_CASE(TA_, TB_) \
    rgemm_kernel<T, TA_, TB_><<<g, 256, 0, c.stream>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, tri)
        if (!tA && !tB) TT_RGEMM_CASE(false, false);
        else if (!tA && tB) TT_RGEMM_CASE(false, true);
        else if (tA && !tB) TT_RGEMM_CASE(true, false);
        else TT_RGEMM_CASE(true, true);
#undef TT_RGEMM_CASE
        TT_LAUNCHED(c);
        return;
    }
    ProfScope ps(c, sizeof(T) == 8 ? "gemm_f64" : "gemm_f32", gemm_flops(M, N, K, tri) * batch,
                 sizeof(T) * ((double)M * K + (double)K * N + 2.0 * M * N) * batch);
    dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM, batch);
    if (grid.y > 65535) throw_status(TT_ERR_ARG, "gemm M too large");
    const long tiles = (long)grid.x * grid.y;
    const long ksteps = (K + GBK - 1) / GBK;
    if (batch == 1 && beta == T(0) && 2 * tiles <= c.sm_count && ksteps >= 16) {
        // few output tiles: split K over about two CTAs per SM (at least 8
        // k-steps each), partials added atomically
        long splits = std::min<long>((2L * c.sm_count + tiles - 1) / tiles, ksteps / 8);
        splits = std::min<long>(splits, 65535);
        const long kchunk = ((ksteps + splits - 1) / splits) * GBK;
        splits = (K + kchunk - 1) / kchunk;
        TT_CUDA(cudaMemset2DAsync(C, ldc * sizeof(T), 0, N * sizeof(T), M, c.stream));
        grid.z = (unsigned)splits;
        launch_gemm<T, T, 2>(c, tA, tB, grid, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, 0, 0, 0, kchunk, tri);
        return;
    }
    launch_gemm<T, T, 0>(c, tA, tB, grid, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sA, sB, sC, K, tri);
}

template <class T, class S>
void gram(Ctx& c, bool rows, int n, long K, const T* X, long ldx, S* G) {
    if constexpr (sizeof(T) == 4 && sizeof(S) == 4) {
        if (sgram(c, rows, n, K, X, ldx, G)) return;
    }
    TT_CUDA(cudaMemsetAsync(G, 0, sizeof(S) * (size_t)n * n, c.stream));
    if (n <= 0 || K <= 0) return;
    const int tiles = (n + GBM - 1) / GBM;
    const int tri = tiles * (tiles + 1) / 2;
    long ksteps = (K + GBK - 1) / GBK;
    long splits = std::max<long>(1, (4L * c.sm_count + tri - 1) / tri);
    splits = std::min<long>(splits, std::max<long>(1, ksteps / 4));
    splits = std::min<long>(splits, 4096);
    long kchunk = ((ksteps + splits - 1) / splits) * GBK;
    splits = (K + kchunk - 1) / kchunk;
    dim3 grid(tiles, tiles, (unsigned)splits);
    ProfScope ps(c, sizeof(T) == 8 ? "gram_f64" : "gram_f32", (double)n * (n + 1) * (double)K,
                 sizeof(T) * (double)n * K + sizeof(S) * (double)n * n);
    // rows: G = X X^T, op(A) = X (n x K), op(B) = X^T  -> tA = false, tB = true
    // cols: G = X^T X, X is K x n: op(A) = X^T -> tA = true, op(B) = X -> tB = false
    launch_gemm<T, S, 1>(c, !rows, rows, grid, n, n, K, T(1), X, ldx, X, ldx, T(0), G, n, 0, 0, 0,
                         kchunk, 0);
}

// ------------------------------------------------------------- reductions
namespace {

template <class C>
__device__ C warp_sum(C v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <class C>
__device__ C block_sum(C v, C* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    C t = (threadIdx.x < nw) ? sh[threadIdx.x] : C(0);
    if (w == 0) t = warp_sum(t);
    if (threadIdx.x == 0) sh[0] = t;
    __syncthreads();
    C r = sh[0];
    __syncthreads();
    return r;
}

template <class T>
__global__ void sumsq_kernel(long n, const T* __restrict__ x, double* out) {
    __shared__ double sh[32];
    double s = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double v = (double)x[i];
        s = fma(v, v, s);
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) atomicAdd(out, s);
}

template <class S>
__global__ void defect_kernel(int n, const S* __restrict__ L, const S* __restrict__ T, double* out) {
    __shared__ double sh[32];
    double a = 0.0, b = 0.0;
    const long nn = (long)n * n;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < nn; e += (long)gridDim.x * blockDim.x) {
        const double t = (double)T[e];
        a = fma(t, t, a);
        const long i = e / n, k = e % n;
        const double l = (double)L[e] - (i == k ? 1.0 : 0.0);
        b = fma(l, l, b);
    }
    a = block_sum(a, sh);
    b = block_sum(b, sh);
    if (threadIdx.x == 0) {
        atomicAdd(out, a);
        atomicAdd(out + 1, b);
    }
}

// E = sym(G) - I from the lower triangle of G, and ||E||_F^2 into *out
template <class T>
__global__ void near_identity_kernel(int n, const T* __restrict__ G, T* __restrict__ E, double* out) {
    __shared__ double sh[32];
    double s = 0.0;
    const long nn = (long)n * n;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < nn; e += (long)gridDim.x * blockDim.x) {
        const long i = e / n, k = e % n;
        const T g = i >= k ? G[e] : G[k * n + i];
        const T v = (i == k) ? g - T(1) : g;
        E[e] = v;
        s = fma((double)v, (double)v, s);
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) atomicAdd(out, s);
}

// S = sum_j a_j E^j, R = sum_j b_j E^j (j = 0..m, E^0 = I); S over E, R may
// alias E2 (every element is read before it is written, by one thread)
template <class T>
__global__ void poly_pair_kernel(int n, int m, T* E, const T* E2, const T* E3, T* R, double a1, double a2,
                                 double a3, double b1, double b2, double b3, const double* e2, double* e2max) {
    // running maximum of ||E||_F^2 over the series passes (non-negative
    // doubles order like their bit patterns)
    if (e2max && blockIdx.x == 0 && threadIdx.x == 0)
        atomicMax(reinterpret_cast<unsigned long long*>(e2max), (unsigned long long)__double_as_longlong(*e2));
    const long nn = (long)n * n;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < nn; e += (long)gridDim.x * blockDim.x) {
        const double id = (e / n == e % n) ? 1.0 : 0.0;
        const double x1 = (double)E[e];
        const double x2 = m >= 2 ? (double)E2[e] : 0.0;
        const double x3 = m >= 3 ? (double)E3[e] : 0.0;
        E[e] = (T)(id + a1 * x1 + a2 * x2 + a3 * x3);
        R[e] = (T)(id + b1 * x1 + b2 * x2 + b3 * x3);
    }
}

}  // namespace

template <class T>
void near_identity(Ctx& c, int n, const T* G, T* E, double* dev_out) {
    TT_CUDA(cudaMemsetAsync(dev_out, 0, sizeof(double), c.stream));
    if (n <= 0) return;
    const long nn = (long)n * n;
    const int blocks = (int)std::min<long>((nn + 255) / 256, 2L * c.sm_count);
    near_identity_kernel<T><<<blocks, 256, 0, c.stream>>>(n, G, E, dev_out);
    TT_LAUNCHED(c);
}

template <class T>
void poly_pair(Ctx& c, int n, int m, T* E, const T* E2, const T* E3, T* R, const double* e2, double* e2max) {
    // Taylor coefficients of (1 + x)^(-1/2) and (1 + x)^(1/2)
    const double a[4] = {1.0, -0.5, 0.375, -0.3125};
    const double b[4] = {1.0, 0.5, -0.125, 0.0625};
    const long nn = (long)n * n;
    if (nn <= 0) return;
    const int blocks = (int)std::min<long>((nn + 255) / 256, 2L * c.sm_count);
    poly_pair_kernel<T><<<blocks, 256, 0, c.stream>>>(n, m, E, E2, E3, R, a[1], m >= 2 ? a[2] : 0.0,
                                                      m >= 3 ? a[3] : 0.0, b[1], m >= 2 ? b[2] : 0.0,
                                                      m >= 3 ? b[3] : 0.0, e2, e2max);
    TT_LAUNCHED(c);
}

template <class T>
void sumsq(Ctx& c, long n, const T* x, double* out) {
    TT_CUDA(cudaMemsetAsync(out, 0, sizeof(double), c.stream));
    if (n <= 0) return;
    int blocks = (int)std::min<long>((n + 255) / 256, 4L * c.sm_count);
    sumsq_kernel<T><<<blocks, 256, 0, c.stream>>>(n, x, out);
    TT_LAUNCHED(c);
}

template <class S>
void inv_and_identity_defect(Ctx& c, int n, const S* L, const S* T, double* out) {
    if (n <= 0) return;
    long nn = (long)n * n;
    int blocks = (int)std::min<long>((nn + 255) / 256, 2L * c.sm_count);
    defect_kernel<S><<<blocks, 256, 0, c.stream>>>(n, L, T, out);
    TT_LAUNCHED(c);
}

// ---------------------------------------------------------- elementwise
namespace {

template <class T>
__global__ void identity_kernel(int n, T* A, long lda) {
    const long nn = (long)n * n;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < nn; e += (long)gridDim.x * blockDim.x) {
        const long i = e / n, k = e % n;
        A[i * lda + k] = (i == k) ? T(1) : T(0);
    }
}

template <class T>
__global__ void scale_kernel(long n, T* x, double alpha) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
        x[e] = (T)((double)x[e] * alpha);
}

template <class Tin, class Tout>
__global__ void convert_kernel(long n, const Tin* __restrict__ x, Tout* __restrict__ y) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
        y[e] = (Tout)x[e];
}

template <class T>
__global__ void transpose_kernel(int rows, int cols, const T* __restrict__ X, T* __restrict__ Y) {
    __shared__ T tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int xr = by + i, xc = bx + threadIdx.x;  // X is cols x rows: X[xr][xc], xr < cols
        if (xr < cols && xc < rows) tile[i][threadIdx.x] = X[(long)xr * rows + xc];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int yr = bx + i, yc = by + threadIdx.x;  // Y[yr][yc] = X[yc][yr]
        if (yr < rows && yc < cols) Y[(long)yr * cols + yc] = tile[threadIdx.x][i];
    }
}

template <class T>
__global__ void scatter_kernel(const BlockList list, int n, long ldb, long ldrow, T* __restrict__ dst) {
    const BlockDesc& bd = list.blk[blockIdx.y];
    const T* src = reinterpret_cast<const T*>(bd.src);
    const long tot = (long)bd.a * n * bd.b;
    const long nb = (long)n * bd.b;
    const T alpha = (T)bd.alpha;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x) {
        const long ia = e / nb, rem = e % nb;
        const long i = rem / bd.b, ib = rem % bd.b;
        dst[bd.dst_off + ia * ldrow + i * ldb + ib] = alpha * src[e];
    }
}

template <class T>
__global__ void axpy_kernel(long n, T alpha, const T* __restrict__ x, T* __restrict__ y) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
        y[e] = fma(alpha, x[e], y[e]);
}

int grid_for(const Ctx& c, long n, int threads = 256) {
    return (int)std::max<long>(1, std::min<long>((n + threads - 1) / threads, 8L * c.sm_count));
}

}  // namespace

template <class T>
void fill_identity(Ctx& c, int n, T* A, long lda) {
    if (n <= 0) return;
    identity_kernel<T><<<grid_for(c, (long)n * n), 256, 0, c.stream>>>(n, A, lda);
    TT_LAUNCHED(c);
}

template <class T>
void scale_inplace(Ctx& c, long n, T* x, double alpha) {
    if (n <= 0) return;
    scale_kernel<T><<<grid_for(c, n), 256, 0, c.stream>>>(n, x, alpha);
    TT_LAUNCHED(c);
}

template <class Tin, class Tout>
void convert(Ctx& c, long n, const Tin* x, Tout* y) {
    if (n <= 0) return;
    convert_kernel<Tin, Tout><<<grid_for(c, n), 256, 0, c.stream>>>(n, x, y);
    TT_LAUNCHED(c);
}

template <class T>
void transpose(Ctx& c, int rows, int cols, const T* X, T* Y) {
    if (rows <= 0 || cols <= 0) return;
    dim3 grid((rows + 31) / 32, (cols + 31) / 32);
    transpose_kernel<T><<<grid, dim3(32, 8), 0, c.stream>>>(rows, cols, X, Y);
    TT_LAUNCHED(c);
}

template <class T>
void scatter_blocks(Ctx& c, const BlockList& list, int n, long dst_ld_b, long dst_ld_row, T* dst, int max_a,
                    int max_b) {
    if (list.count <= 0) return;
    long per = (long)max_a * n * max_b;
    dim3 grid((unsigned)std::max<long>(1, std::min<long>((per + 255) / 256, 1024)), list.count);
    ProfScope ps(c, "tt_add_scatter", 0.0, 2.0 * sizeof(T) * per * list.count);
    scatter_kernel<T><<<grid, 256, 0, c.stream>>>(list, n, dst_ld_b, dst_ld_row, dst);
    TT_LAUNCHED(c);
}

template <class T>
void axpy(Ctx& c, long n, double alpha, const T* x, T* y) {
    if (n <= 0) return;
    axpy_kernel<T><<<grid_for(c, n), 256, 0, c.stream>>>(n, (T)alpha, x, y);
    TT_LAUNCHED(c);
}

// ------------------------------------------------- explicit instantiations
#define TT_INST_T(T)                                                                             \
    template void gemm<T>(Ctx&, bool, bool, int, int, int, T, const T*, long, const T*, long, T, T*, \
                          long, int, long, long, long, int);                                       \
    template void sumsq<T>(Ctx&, long, const T*, double*);                                       \
    template void fill_identity<T>(Ctx&, int, T*, long);                                         \
    template void scale_inplace<T>(Ctx&, long, T*, double);                                      \
    template void transpose<T>(Ctx&, int, int, const T*, T*);                                    \
    template void scatter_blocks<T>(Ctx&, const BlockList&, int, long, long, T*, int, int);      \
    template void axpy<T>(Ctx&, long, double, const T*, T*);                                     \
    template void inv_and_identity_defect<T>(Ctx&, int, const T*, const T*, double*);             \
    template void near_identity<T>(Ctx&, int, const T*, T*, double*);                            \
    template void poly_pair<T>(Ctx&, int, int, T*, const T*, const T*, T*, const double*, double*);
TT_INST_T(float)
TT_INST_T(double)
template void gram<double, double>(Ctx&, bool, int, long, const double*, long, double*);
template void gram<float, float>(Ctx&, bool, int, long, const float*, long, float*);
template void convert<double, float>(Ctx&, long, const double*, float*);
template void convert<float, double>(Ctx&, long, const float*, double*);

}  // namespace ttgb
