// Split-TF32 GEMM on the 5th-generation tensor cores: C = A op(B) with FP32
// operands, each split into round-to-nearest TF32 parts, kind::tf32 MMAs with
// FP32 accumulation in TMEM.  Three parts x = hi + mid + lo and the six
// products hh, hm, mh, hl, lh, mm leave only terms below 2^-33 |a||b| out
// (FP32-level products); two parts x = hi + lo and the products hh, hl, lh
// leave ~2^-22.  These are the GEMMs of TT-round that produce core values
// (apply Q = L^{-1} X and absorb core <- core L), where plain TF32 (10-bit
// mantissa) would perturb the represented tensor by ~1e-3.
//
// A is M x K row-major (K contiguous).  B is either N x K row-major
// ("T": C = A B^T) or K x N row-major ("N": C = A B, N contiguous).  One CTA
// computes a 128 x 128 tile of C: warp 0 streams raw FP32 tiles with TMA into
// a 2-deep staging ring; warps 2-5 split them into TF32 hi/lo parts written
// in the 128-byte-swizzled K-major layout the MMA reads (transposing B when it
// is N-major) into a 2-deep operand ring; warp 1 issues the MMAs; warps 2-5
// then read the accumulator from TMEM and store C.  Every wait is bounded.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "internal.h"
#include "tc_common.cuh"

namespace ttgb {

namespace {

constexpr int BM = 128, BN = 128, BK = 32;
constexpr int TILE = BM * BK * 4;  // 16 KB, one operand tile
constexpr int NSTG = 2;
constexpr uint32_t TMEM_COLS = 256;  // two 128-column accumulators
constexpr long long WAIT_LIMIT = 4000000000LL;

constexpr int NOP_MAX = 2;

struct __align__(8) GemmCtl {
    uint64_t stg_full[NSTG], stg_empty[NSTG];
    uint64_t op_full[NOP_MAX], op_empty[NOP_MAX];
    uint64_t acc_full[2], acc_empty[2];
    uint64_t done;
    uint32_t tmem_base;
};

__device__ __forceinline__ uint32_t rna_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// three-way split x = hi + mid + lo, each round-to-nearest TF32; the
// remainder is below 2^-33 |x|
__device__ __forceinline__ void split4x3(const float4 v, float4& hi, float4& mi, float4& lo) {
    float h[4], m[4], l[4];
    const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        h[i] = __uint_as_float(rna_tf32(x[i]));
        const float r = x[i] - h[i];
        m[i] = __uint_as_float(rna_tf32(r));
        l[i] = __uint_as_float(rna_tf32(r - m[i]));
    }
    hi = make_float4(h[0], h[1], h[2], h[3]);
    mi = make_float4(m[0], m[1], m[2], m[3]);
    lo = make_float4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ void split4(const float4 v, float4& hi, float4& lo) {
    const float h0 = __uint_as_float(rna_tf32(v.x)), h1 = __uint_as_float(rna_tf32(v.y));
    const float h2 = __uint_as_float(rna_tf32(v.z)), h3 = __uint_as_float(rna_tf32(v.w));
    hi = make_float4(h0, h1, h2, h3);
    lo = make_float4(__uint_as_float(rna_tf32(v.x - h0)), __uint_as_float(rna_tf32(v.y - h1)),
                     __uint_as_float(rna_tf32(v.z - h2)), __uint_as_float(rna_tf32(v.w - h3)));
}

// writes the NS parts of v to the same offset of NS consecutive tiles
template <int NS>
__device__ __forceinline__ void store_parts(const float4 v, unsigned char* dst) {
    if (NS == 3) {
        float4 h, m, l;
        split4x3(v, h, m, l);
        *reinterpret_cast<float4*>(dst) = h;
        *reinterpret_cast<float4*>(dst + TILE) = m;
        *reinterpret_cast<float4*>(dst + 2 * TILE) = l;
    } else {
        float4 h, l;
        split4(v, h, l);
        *reinterpret_cast<float4*>(dst) = h;
        *reinterpret_cast<float4*>(dst + TILE) = l;
    }
}

// byte offset of the 16-byte chunk c4 of row r in a 128-byte-swizzled tile
__device__ __forceinline__ int sw128(int r, int c4) { return r * 128 + ((c4 ^ (r & 7)) << 4); }

// NS = 2: x = hi + lo, products hi*hi + hi*lo + lo*hi (3 MMAs per k-step)
// NS = 3: x = hi + mid + lo, products hh + hm + mh + hl + lh + mm (6 MMAs)
template <bool BT, int NS>
__global__ void __launch_bounds__(192, 1)
gemm3_tf32_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M, int N,
                  int K, float* __restrict__ Cm, long ldc, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    // operand ring first (1024-aligned tiles): [NOP][A parts.., B parts..]
    constexpr int NOP = (NS == 3) ? 1 : 2;
    constexpr int OPT = 2 * NS;  // tiles per operand stage
    unsigned char* opr = base;
    unsigned char* stg = opr + NOP * OPT * TILE;  // [NSTG][A raw, B raw]
    GemmCtl* ctl = reinterpret_cast<GemmCtl*>(stg + NSTG * 2 * TILE);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int nk = (K + BK - 1) / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTG; ++s) {
            tc::mbar_init(&ctl->stg_full[s], 1);
            tc::mbar_init(&ctl->stg_empty[s], 128);
        }
        for (int s = 0; s < NOP; ++s) {
            tc::mbar_init(&ctl->op_full[s], 128);
            tc::mbar_init(&ctl->op_empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(&ctl->acc_full[s], 1);
            tc::mbar_init(&ctl->acc_empty[s], 128);
        }
        tc::mbar_init(&ctl->done, 1);
        tc::fence_barrier_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(&ctl->tmem_base, TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = ctl->tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            tc::prefetch_tmap(&mapA);
            tc::prefetch_tmap(&mapB);
            bool ok = true;
            int issued = 0;
            for (int it = 0; it < nk; ++it) {
                const int s = it % NSTG;
                if (!tc::mbar_wait_bounded(&ctl->stg_empty[s], ((it / NSTG) & 1) ^ 1, WAIT_LIMIT)) { ok = false; break; }
                unsigned char* a = stg + s * 2 * TILE;
                tc::mbar_arrive_expect_tx(&ctl->stg_full[s], 2 * TILE);
                tc::tma_load_2d(a, &mapA, &ctl->stg_full[s], it * BK, m0);
                if (BT) tc::tma_load_2d(a + TILE, &mapB, &ctl->stg_full[s], it * BK, n0);
                else tc::tma_load_2d(a + TILE, &mapB, &ctl->stg_full[s], n0, it * BK);
                ++issued;
            }
            if (!ok) {
                atomicExch(err, 1);
                for (int it = max(0, issued - NSTG); it < issued; ++it)
                    tc::mbar_wait_bounded(&ctl->stg_full[it % NSTG], (it / NSTG) & 1, WAIT_LIMIT);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_tf32(BM, BN);
            bool ok = true;
            for (int it = 0; it < nk; ++it) {
                const int o = it % NOP, ab = it & 1;
                // accumulator buffer ab must have been read back by the promoters
                if (!tc::mbar_wait_bounded(&ctl->acc_empty[ab], ((it >> 1) & 1) ^ 1, WAIT_LIMIT)) { ok = false; break; }
                if (!tc::mbar_wait_bounded(&ctl->op_full[o], (it / NOP) & 1, WAIT_LIMIT)) { ok = false; break; }
                tc::tc_fence_after();
                const uint32_t dacc = tmem + ab * 128;
                // A parts at tiles 0..NS-1, B parts at NS..2NS-1: 0 = hi, 1 = lo (NS = 2)
                // or 0 = hi, 1 = mid, 2 = lo (NS = 3)
                const uint32_t a0 = tc::smem_u32(opr + o * OPT * TILE);
                const uint32_t b0 = a0 + NS * TILE;
                // each k-step starts a fresh partial sum (promoted to FP32
                // registers by the converter warps).  Products go in order of
                // increasing magnitude, the hi*hi ones last, so that the
                // accumulator's rounding acts on small partial sums for as
                // long as possible.
                auto ad = [&](int part, int kk) { return tc::sdesc_kmajor_sw128(a0 + part * TILE + kk * 32); };
                auto bd = [&](int part, int kk) { return tc::sdesc_kmajor_sw128(b0 + part * TILE + kk * 32); };
                uint32_t accf = 0u;
                if (NS == 3) {
#pragma unroll
                    for (int kk = 0; kk < BK / 8; ++kk) {
                        tc::mma_tf32(dacc, ad(1, kk), bd(1, kk), idesc, accf);  // mid * mid
                        accf = 1u;
                        tc::mma_tf32(dacc, ad(0, kk), bd(2, kk), idesc, 1u);    // hi * lo
                        tc::mma_tf32(dacc, ad(2, kk), bd(0, kk), idesc, 1u);    // lo * hi
                    }
                }
#pragma unroll
                for (int kk = 0; kk < BK / 8; ++kk) {
                    tc::mma_tf32(dacc, ad(0, kk), bd(1, kk), idesc, accf);      // hi * mid (or lo)
                    accf = 1u;
                    tc::mma_tf32(dacc, ad(1, kk), bd(0, kk), idesc, 1u);        // mid (or lo) * hi
                }
#pragma unroll
                for (int kk = 0; kk < BK / 8; ++kk) tc::mma_tf32(dacc, ad(0, kk), bd(0, kk), idesc, 1u);  // hi * hi
                tc::mma_commit(&ctl->op_empty[o]);
                tc::mma_commit(&ctl->acc_full[ab]);
            }
            if (!ok) atomicExch(err, 1);
            tc::mma_commit(&ctl->done);
        }
    } else {
        // converters / promoters (warps 2..5, 128 threads): split stage it
        // into TF32 parts, then add the partial sum of k-step it-1 from TMEM
        // into FP32 registers (round-to-nearest); finally store C
        const int t = threadIdx.x - 64;
        const int q = warp & 3;  // TMEM lane quarter this warp may read
        float acc[BN];
#pragma unroll
        for (int j = 0; j < BN; ++j) acc[j] = 0.f;
        bool ok = true;
        auto promote = [&](int j) -> bool {
            const int ab = j & 1;
            const bool g = __all_sync(0xffffffffu, tc::mbar_wait_bounded(&ctl->acc_full[ab], (j >> 1) & 1, WAIT_LIMIT));
            if (!g) return false;
            tc::tc_fence_after();
#pragma unroll
            for (int c = 0; c < BN / 32; ++c) {
                float v[32];
                __syncwarp();
                tc::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + ab * 128 + c * 32, v);
#pragma unroll
                for (int i = 0; i < 32; ++i) acc[c * 32 + i] += v[i];
            }
            tc::tc_fence_before();
            tc::mbar_arrive(&ctl->acc_empty[ab]);
            return true;
        };
        for (int it = 0; it < nk && ok; ++it) {
            const int s = it % NSTG, o = it % NOP;
            const bool g1 = tc::mbar_wait_bounded(&ctl->stg_full[s], (it / NSTG) & 1, WAIT_LIMIT);
            const bool g2 = g1 && tc::mbar_wait_bounded(&ctl->op_empty[o], ((it / NOP) & 1) ^ 1, WAIT_LIMIT);
            ok = __all_sync(0xffffffffu, g1 && g2);
            if (!ok) break;
            const unsigned char* sa = stg + s * 2 * TILE;
            const unsigned char* sb = sa + TILE;
            unsigned char* a0 = opr + o * OPT * TILE;
            unsigned char* b0 = a0 + NS * TILE;
            // A (and B when K-major): staging [128 rows][32 k], 8 chunks of 4 per row
#pragma unroll
            for (int qq = 0; qq < 8; ++qq) {
                const int idx = qq * 128 + t;
                const int r = idx >> 3, c4 = idx & 7;
                const int off = sw128(r, c4);
                store_parts<NS>(*reinterpret_cast<const float4*>(sa + r * 128 + c4 * 16), a0 + off);
                if (BT) store_parts<NS>(*reinterpret_cast<const float4*>(sb + r * 128 + c4 * 16), b0 + off);
            }
            if (!BT) {
                // B N-major: staging [32 k][128 n]; operand row n holds k = 0..31
#pragma unroll
                for (int qq = 0; qq < 8; ++qq) {
                    const int idx = qq * 128 + t;
                    const int nn = idx & 127, c4 = idx >> 7;
                    const float* col = reinterpret_cast<const float*>(sb) + (c4 * 4) * BN + nn;
                    store_parts<NS>(make_float4(col[0], col[BN], col[2 * BN], col[3 * BN]), b0 + sw128(nn, c4));
                }
            }
            // every converter thread makes its own generic-proxy writes visible
            // to the async proxy (tcgen05.mma) and arrives itself
            fence_proxy_async();
            tc::mbar_arrive(&ctl->op_full[o]);
            tc::mbar_arrive(&ctl->stg_empty[s]);
            if (it >= 1) ok = promote(it - 1);
        }
        if (ok) ok = promote(nk - 1);
        if (!ok && lane == 0) atomicExch(err, 1);
        int e = 0;
        if (lane == 0) e = *(volatile int*)err;
        e = __shfl_sync(0xffffffffu, e, 0);
        if (ok && e == 0) {
            const int row = m0 + q * 32 + lane;
            if (row < M) {
                float* dst = Cm + (long)row * ldc + n0;
                if (n0 + BN <= N && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
#pragma unroll
                    for (int j = 0; j < BN; j += 4)
                        *reinterpret_cast<float4*>(dst + j) = make_float4(acc[j], acc[j + 1], acc[j + 2], acc[j + 3]);
                } else {
#pragma unroll
                    for (int j = 0; j < BN; ++j)
                        if (n0 + j < N) dst[j] = acc[j];
                }
            }
        }
    }
    // the MMA issuer makes sure its MMAs have finished before TMEM is freed
    if (warp == 1 && lane == 0) tc::mbar_wait_bounded(&ctl->done, 0, WAIT_LIMIT);
    __syncwarp();
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, TMEM_COLS);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

bool make_map(CUtensorMap* map, const float* ptr, long inner, long outer, long ld, int box_inner, int box_outer) {
    auto enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
    cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)ptr, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool gemm_tc3_tf32(Ctx& c, bool bT, int M, int N, int K, const float* A, long lda, const float* B, long ldb,
                   float* C, long ldc, int nsplit) {
    if (M <= 0 || N <= 0 || K <= 0 || (nsplit != 2 && nsplit != 3)) return false;
    auto aligned = [](const void* p, long ld) { return ((uintptr_t)p & 15) == 0 && (ld * 4) % 16 == 0; };
    if (!aligned(A, lda) || !aligned(B, ldb)) return false;
    if (lda < K || (bT ? ldb < K : ldb < N) || ldc < N) return false;
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, K, M, lda, BK, BM)) return false;
    if (bT) {
        if (!make_map(&mb, B, K, N, ldb, BK, BN)) return false;
    } else {
        if (!make_map(&mb, B, N, K, ldb, BN, BK)) return false;
    }
    const dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    if (grid.y > 65535) return false;
    const int nop = (nsplit == 3) ? 1 : 2;
    const size_t smem = 1024 + (size_t)nop * 2 * nsplit * TILE + NSTG * 2 * TILE + sizeof(GemmCtl) + 64;
    static std::atomic<bool> attr[2][2];
    const int si = nsplit - 2;
    if (bT && si) set_smem_once(attr[1][1], gemm3_tf32_kernel<true, 3>, (int)smem);
    else if (bT) set_smem_once(attr[1][0], gemm3_tf32_kernel<true, 2>, (int)smem);
    else if (si) set_smem_once(attr[0][1], gemm3_tf32_kernel<false, 3>, (int)smem);
    else set_smem_once(attr[0][0], gemm3_tf32_kernel<false, 2>, (int)smem);
    ProfScope ps(c, nsplit == 3 ? "gemm_tf32x6_tc" : "gemm_tf32x3_tc", 2.0 * M * (double)N * K,
                 4.0 * ((double)M * K + (double)K * N + (double)M * N));
    if (bT && si) gemm3_tf32_kernel<true, 3><<<grid, 192, smem, c.stream>>>(ma, mb, M, N, K, C, ldc, c.tc_err);
    else if (bT) gemm3_tf32_kernel<true, 2><<<grid, 192, smem, c.stream>>>(ma, mb, M, N, K, C, ldc, c.tc_err);
    else if (si) gemm3_tf32_kernel<false, 3><<<grid, 192, smem, c.stream>>>(ma, mb, M, N, K, C, ldc, c.tc_err);
    else gemm3_tf32_kernel<false, 2><<<grid, 192, smem, c.stream>>>(ma, mb, M, N, K, C, ldc, c.tc_err);
    TT_LAUNCHED(c);
    return true;
}

}  // namespace ttgb
