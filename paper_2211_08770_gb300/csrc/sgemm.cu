// FP32 CUDA-core GEMM and split-K Gram for the products of TT-round that stay
// in FP32 arithmetic: the applies X <- T X and X <- X T^T, the absorbs of the
// R factors into the neighbouring core, the second Cholesky QR pass's Gram
// and the contractions of the TT dot (Section 2).
//
// 128 x 128 output tile per CTA of 256 threads, 8 x 8 outputs per thread
// (two 4 x 4 quadrants 64 apart, so a warp's shared-memory reads are 16-byte
// broadcasts or conflict-free), BK = 8 with the next k-slab loaded into
// registers while the current one is multiplied (double-buffered shared
// memory, one barrier per slab).  The products are packed FP32x2 FMAs (two
// accumulators per instruction: the kernel is issue-bound), and in a partial
// edge tile the warps whose outputs lie beyond the edge skip them (r = 400
// leaves 112 of the last tile's 128 rows or columns empty).  Operands enter with 16-byte loads; the
// row-major M x K (or N x K) side is transposed into k-major shared memory on
// the way, with the tile rows padded by four floats so the scattered stores
// do not collide.  Requires 16-byte aligned pointers and leading dimensions
// that are multiples of four floats; other layouts take the 64 x 64 kernel.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "internal.h"

namespace ttgb {

namespace {

constexpr int SBM = 128, SBN = 128, SBK = 8, SPAD = 4;

// op(X) is rows x K; !T: X is rows x K row-major (k contiguous); T: X is
// K x rows row-major (rows contiguous).  Thread t loads one float4:
//  !T: row r0 + t / 2, k = k0 + 4 (t % 2) .. + 3
//   T: k = k0 + t / 32, row r0 + 4 (t % 32) .. + 3
template <bool T>
__device__ __forceinline__ float4 load_slab(const float* __restrict__ X, long ld, int rows, long kend, int r0,
                                            long k0) {
    const int t = threadIdx.x;
    float e[4];
    if (!T) {
        const long r = r0 + (t >> 1);
        const long k = k0 + 4 * (t & 1);
        if (r < rows && k + 3 < kend) return *reinterpret_cast<const float4*>(X + r * ld + k);
#pragma unroll
        for (int i = 0; i < 4; ++i) e[i] = (r < rows && k + i < kend) ? X[r * ld + k + i] : 0.f;
    } else {
        const long k = k0 + (t >> 5);
        const long r = r0 + 4 * (t & 31);
        if (k < kend && r + 3 < rows) return *reinterpret_cast<const float4*>(X + k * ld + r);
#pragma unroll
        for (int i = 0; i < 4; ++i) e[i] = (k < kend && r + i < rows) ? X[k * ld + r + i] : 0.f;
    }
    return make_float4(e[0], e[1], e[2], e[3]);
}

// store the slab into k-major shared memory S[k][row] (row stride SBM + SPAD)
template <bool T>
__device__ __forceinline__ void store_slab(float* S, const float4 v) {
    const int t = threadIdx.x;
    constexpr int LD = SBM + SPAD;
    if (!T) {
        const int r = t >> 1, k = 4 * (t & 1);
        S[(k + 0) * LD + r] = v.x;
        S[(k + 1) * LD + r] = v.y;
        S[(k + 2) * LD + r] = v.z;
        S[(k + 3) * LD + r] = v.w;
    } else {
        const int k = t >> 5, r = 4 * (t & 31);
        *reinterpret_cast<float4*>(S + k * LD + r) = v;
    }
}

// acc (two adjacent FP32 accumulators) += a * (b.x, b.y): one packed
// FP32x2 FMA (sm_100 and later), half the issue slots of two FFMAs; the same
// rounding as two fmaf
__device__ __forceinline__ void fma2(float& c0, float& c1, float a, float b0, float b1) {
    unsigned long long cc, ap, bp;
    asm("mov.b64 %0, {%1, %2};" : "=l"(cc) : "f"(c0), "f"(c1));
    asm("mov.b64 %0, {%1, %1};" : "=l"(ap) : "f"(a));
    asm("mov.b64 %0, {%1, %2};" : "=l"(bp) : "f"(b0), "f"(b1));
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(cc) : "l"(ap), "l"(bp));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(c0), "=f"(c1) : "l"(cc));
}

// C (M x N) = alpha op(A) op(B) + beta C   (MODE 0, blockIdx.z = batch)
// C += op(A) op(B) on lower tiles, split-K (MODE 1, blockIdx.z = K split)
// CW: a warp covers 2 column groups x 16 row groups (else 16 x 2), so a
// warp whose outputs all fall beyond N (CW) or M (!CW) in a partial edge
// tile skips the products (it still stages its share of the operands).
template <bool TA, bool TB, int MODE, bool CW>
__global__ void __launch_bounds__(256, 2)
sgemm_kernel(int M, int N, long K, float alpha, const float* __restrict__ A, long lda, const float* __restrict__ B,
             long ldb, float beta, float* __restrict__ C, long ldc, long sA, long sB, long sC, long kchunk, int tri) {
    constexpr int LD = SBM + SPAD;
    __shared__ __align__(16) float As[2][SBK * LD];
    __shared__ __align__(16) float Bs[2][SBK * LD];
    const int tid = threadIdx.x;
    const int tx = CW ? tid >> 4 : tid & 15, ty = CW ? tid & 15 : tid >> 4;
    // a lower-triangular op(A) gives the last row tiles the longest
    // k-ranges: those are dispatched first (blocks start in x-then-y order),
    // so the short tiles fill the end of the launch instead of the long ones
    const int by = (MODE == 0 && (tri & TRI_A_LOWER)) ? (int)(gridDim.y - 1 - blockIdx.y) : (int)blockIdx.y;
    const int m0 = by * SBM, n0 = blockIdx.x * SBN;
    // outputs 4 t.. precede 64 + 4 t.., so the first group decides
    const bool live = CW ? (n0 + 4 * tx < N) : (m0 + 4 * ty < M);
    long kbeg = 0, kend = K;
    if (MODE == 0) {
        A += blockIdx.z * sA;
        B += blockIdx.z * sB;
        C += blockIdx.z * sC;
        if (tri_skip_tile(tri, m0, n0, SBM)) return;
        tri_krange(tri, m0, n0, SBM, SBN, kbeg, kend);  // tile multiples of SBK
    } else {
        if (blockIdx.x > blockIdx.y) return;  // upper tiles of the symmetric result
        kbeg = (long)blockIdx.z * kchunk;
        kend = min(K, kbeg + kchunk);
        if (kbeg >= kend) return;
    }
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    float4 ra = load_slab<TA>(A, lda, M, kend, m0, kbeg);
    float4 rb = load_slab<!TB>(B, ldb, N, kend, n0, kbeg);
    store_slab<TA>(As[0], ra);
    store_slab<!TB>(Bs[0], rb);
    __syncthreads();
    int buf = 0;
    for (long k0 = kbeg; k0 < kend; k0 += SBK) {
        const bool more = k0 + SBK < kend;
        if (more) {
            ra = load_slab<TA>(A, lda, M, kend, m0, k0 + SBK);
            rb = load_slab<!TB>(B, ldb, N, kend, n0, k0 + SBK);
        }
        const float* a_s = As[buf];
        const float* b_s = Bs[buf];
        if (live) {
#pragma unroll
            for (int kk = 0; kk < SBK; ++kk) {
                const float4 a0 = *reinterpret_cast<const float4*>(a_s + kk * LD + 4 * ty);
                const float4 a1 = *reinterpret_cast<const float4*>(a_s + kk * LD + 64 + 4 * ty);
                const float4 b0 = *reinterpret_cast<const float4*>(b_s + kk * LD + 4 * tx);
                const float4 b1 = *reinterpret_cast<const float4*>(b_s + kk * LD + 64 + 4 * tx);
                const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; j += 2) fma2(acc[i][j], acc[i][j + 1], av[i], bv[j], bv[j + 1]);
            }
        }
        if (more) {
            store_slab<TA>(As[buf ^ 1], ra);
            store_slab<!TB>(Bs[buf ^ 1], rb);
        }
        __syncthreads();
        buf ^= 1;
    }
    // rows m0 + 4 ty + {0..3} and + 64; columns n0 + 4 tx + {0..3} and + 64
    const bool cvec = ((ldc & 3) == 0) && (((uintptr_t)C & 15) == 0);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const long gm = m0 + 4 * ty + (i & 3) + (i >= 4 ? 64 : 0);
        if (gm >= M) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const long gn = n0 + 4 * tx + 64 * h;
            float* cp = C + gm * ldc + gn;
            const float* v = &acc[i][4 * h];
            if (MODE == 0) {
                float o[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    o[e] = alpha * v[e];
                    if (beta != 0.f && gn + e < N) o[e] = fmaf(beta, cp[e], o[e]);
                }
                if ((tri & TRI_C_LOWER) && gn + 3 > gm) {  // lower triangle only
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (gn + e < N && gn + e <= gm) cp[e] = o[e];
                } else if (gn + 3 < N && cvec) {
                    *reinterpret_cast<float4*>(cp) = make_float4(o[0], o[1], o[2], o[3]);
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (gn + e < N) cp[e] = o[e];
                }
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (gn + e < N) atomicAdd(cp + e, v[e]);
            }
        }
    }
}

template <int MODE>
void launch_sgemm(Ctx& c, bool tA, bool tB, dim3 grid, int M, int N, long K, float alpha, const float* A, long lda,
                  const float* B, long ldb, float beta, float* C, long ldc, long sA, long sB, long sC, long kchunk,
                  int tri) {
    // skip along the dimension whose edge tile wastes more of its width
    const int wm = (int)(grid.y * SBM - M), wn = (int)(grid.x * SBN - N);
    const bool cw = MODE == 0 && wn > wm;
#define TT_SGEMM_CASE(TA_, TB_)                                                                                  \
    do {                                                                                                         \
        if constexpr (MODE == 0)                                                                                 \
            if (cw) {                                                                                            \
                sgemm_kernel<TA_, TB_, MODE, true><<<grid, 256, 0, c.stream>>>(M, N, K, alpha, A, lda, B, ldb,   \
                                                                               beta, C, ldc, sA, sB, sC, kchunk, \
                                                                               tri);                             \
                break;                                                                                           \
            }                                                                                                    \
            sgemm_kernel<TA_, TB_, MODE, false><<<grid, 256, 0, c.stream>>>(M, N, K, alpha, A, lda, B, ldb,      \
                                                                            beta, C, ldc, sA, sB, sC, kchunk,    \
                                                                            tri);                                \
    } while (0)
    if (!tA && !tB) TT_SGEMM_CASE(false, false);
    else if (!tA && tB) TT_SGEMM_CASE(false, true);
    else if (tA && !tB) TT_SGEMM_CASE(true, false);
    else TT_SGEMM_CASE(true, true);
#undef TT_SGEMM_CASE
    TT_LAUNCHED(c);
}

inline bool al16(const void* p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace

bool sgemm(Ctx& c, bool tA, bool tB, int M, int N, int K, float alpha, const float* A, long lda, const float* B,
           long ldb, float beta, float* C, long ldc, int batch, long sA, long sB, long sC, int tri) {
    if ((lda & 3) || (ldb & 3) || !al16(A) || !al16(B)) return false;
    if (batch > 1 && ((sA & 3) || (sB & 3))) return false;
    dim3 grid((N + SBN - 1) / SBN, (M + SBM - 1) / SBM, batch);
    if (grid.y > 65535) return false;
    ProfScope ps(c, "sgemm_f32", gemm_flops(M, N, K, tri) * batch,
                 sizeof(float) * ((double)M * K + (double)K * N + 2.0 * M * N) * batch);
    launch_sgemm<0>(c, tA, tB, grid, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sA, sB, sC, K, tri);
    return true;
}

bool sgram(Ctx& c, bool rows, int n, long K, const float* X, long ldx, float* G) {
    if ((ldx & 3) || !al16(X)) return false;
    TT_CUDA(cudaMemsetAsync(G, 0, sizeof(float) * (size_t)n * n, c.stream));
    if (n <= 0 || K <= 0) return true;
    const int tiles = (n + SBM - 1) / SBM;
    const int tri = tiles * (tiles + 1) / 2;
    const long ksteps = (K + SBK - 1) / SBK;
    // about two CTAs per SM over the lower tiles, at least 32 k-slabs each
    long splits = std::max<long>(1, (2L * c.sm_count + tri - 1) / tri);
    splits = std::min<long>(splits, std::max<long>(1, ksteps / 32));
    splits = std::min<long>(splits, 4096);
    const long kchunk = ((ksteps + splits - 1) / splits) * SBK;
    splits = (K + kchunk - 1) / kchunk;
    dim3 grid(tiles, tiles, (unsigned)splits);
    ProfScope ps(c, "sgram_f32", (double)n * (n + 1) * (double)K, sizeof(float) * ((double)n * K + (double)n * n));
    // rows: G = X X^T, op(A) = X (n x K), op(B) = X^T: tA = false, tB = true
    // cols: G = X^T X with X K x n: op(A) = X^T: tA = true; op(B) = X: tB = false
    launch_sgemm<1>(c, !rows, rows, grid, n, n, K, 1.f, X, ldx, X, ldx, 0.f, G, n, 0, 0, 0, kchunk, 0);
    return true;
}

}  // namespace ttgb
