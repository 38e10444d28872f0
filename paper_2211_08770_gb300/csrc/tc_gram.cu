// Gram matrix G = X X^T of the rows of an FP32 matrix X (n x K, row-major,
// K contiguous) on the 5th-generation tensor cores (tcgen05, kind::tf32,
// FP32 accumulation in TMEM): the Gram step of the Cholesky QR passes of the
// right-to-left TT-rounding sweep.
//
// One CTA computes one 128 x 128 tile (tile_i >= tile_j: lower tiles only,
// G is symmetric) over one chunk of K (split-K) and adds it atomically into
// G.  Warp 0 issues TMA loads of 128 x 32 FP32 boxes (128-byte swizzle) into
// a 5-stage ring; warp 1 allocates 128 TMEM columns and issues 4 MMAs of
// 128 x 128 x 8 per stage; warps 2-5 read the accumulator back with
// tcgen05.ld and add it into G through shared memory, one row segment per
// warp instruction.  Every mbarrier wait is bounded (the context's limit, about
// 2 s by default); a timeout sets *err and the CTA winds down: it stops
// issuing work, lets the copies already issued land and waits for its MMAs
// (both with the long limit), and always frees TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "internal.h"
#include "tc_common.cuh"

namespace ttgb {

namespace {

constexpr int TB = 128;           // tile rows (= MMA M = N)
constexpr int TK = 32;            // fp32 per 128-byte swizzled row
constexpr int STAGES = 5;
constexpr int TILE_BYTES = TB * TK * 4;  // 16 KB
constexpr uint32_t TMEM_COLS = 128;
constexpr long long WAIT_LIMIT = 4000000000LL;  // ~2 s of SM cycles

struct __align__(8) GramSmem {
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    uint64_t done;
    uint32_t tmem_base;
};

// Adds the 32 x 128 block of this CTA's accumulator held in TMEM lanes
// [32 q, 32 q + 32) (taddr = its first column) into G[row0 + i][col0 + j]
// (n x n, row-major), clipped to n.  Each 32 x 32 piece goes through a
// padded shared-memory stage (stg: 32 x 33 floats of this warp), so that one
// warp instruction adds 32 consecutive floats of one row (one cache line)
// instead of one float of 32 rows.
__device__ __forceinline__ void add_block_rows(uint32_t taddr, float* stg, float* __restrict__ G, int n, int row0,
                                               int col0, int lane) {
    float v[32];
#pragma unroll 1
    for (int c = 0; c < TB / 32; ++c) {
        __syncwarp();
        tc::tmem_ld32(taddr + c * 32, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) stg[lane * 33 + j] = v[j];
        __syncwarp();
        const int col = col0 + c * 32 + lane;
#pragma unroll 4
        for (int i = 0; i < 32; ++i) {
            const int row = row0 + i;
            if (row < n && col < n) atomicAdd(&G[(long)row * n + col], stg[i * 33 + lane]);
        }
    }
}

__global__ void __launch_bounds__(192, 1)
gram_tf32_kernel(const __grid_constant__ CUtensorMap tmap, int n, long K, int ntiles, long kchunk_steps,
                 float* __restrict__ G, int* __restrict__ err, long long limit) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned operand ring, control block after it
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* ring = base;  // STAGES x (A 16 KB, B 16 KB)
    GramSmem* ctl = reinterpret_cast<GramSmem*>(ring + STAGES * 2 * TILE_BYTES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // decode (tile_i, tile_j) with tile_i >= tile_j, and the K split
    const int ntri = ntiles * (ntiles + 1) / 2;
    const int pair = blockIdx.x % ntri;
    const long split = blockIdx.x / ntri;
    int ti = 0;
    while ((ti + 1) * (ti + 2) / 2 <= pair) ++ti;
    const int tj = pair - ti * (ti + 1) / 2;
    const bool diag = (ti == tj);
    const long ksteps_total = (K + TK - 1) / TK;
    const long ks0 = split * kchunk_steps;
    const long ks1 = min(ksteps_total, ks0 + kchunk_steps);
    const int nsteps = (int)max(0L, ks1 - ks0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&ctl->full[s], 1);
            tc::mbar_init(&ctl->empty[s], 1);
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
    bool ok = true;

    if (warp == 0) {
        if (lane == 0 && nsteps > 0) {
            tc::prefetch_tmap(&tmap);
            const uint32_t bytes = diag ? TILE_BYTES : 2 * TILE_BYTES;
            int issued = 0;
            for (int it = 0; it < nsteps; ++it) {
                const int s = it % STAGES;
                const uint32_t ph = (it / STAGES) & 1;
                if (!tc::mbar_wait_bounded(&ctl->empty[s], ph ^ 1, limit)) { ok = false; break; }
                unsigned char* a = ring + s * 2 * TILE_BYTES;
                tc::mbar_arrive_expect_tx(&ctl->full[s], bytes);
                const int kx = (int)((ks0 + it) * TK);
                tc::tma_load_2d(a, &tmap, &ctl->full[s], kx, ti * TB);
                if (!diag) tc::tma_load_2d(a + TILE_BYTES, &tmap, &ctl->full[s], kx, tj * TB);
                ++issued;
            }
            if (!ok) atomicExch(err, 1);
            // every copy issued lands before the CTA can exit, also when the
            // MMA warp gave up consuming them: issuing step it + STAGES
            // waited for step it to be consumed (its copy landed), so only
            // the last STAGES issued can still be in flight.  A completed
            // phase answers at once; the wait keeps the long limit whatever
            // the context's limit is.
            for (int it = max(0, issued - STAGES); it < issued; ++it)
                tc::mbar_wait_bounded(&ctl->full[it % STAGES], (it / STAGES) & 1, WAIT_LIMIT);
        }
    } else if (warp == 1) {
        if (lane == 0 && nsteps > 0) {
            constexpr uint32_t idesc = tc::idesc_tf32(TB, TB);
            for (int it = 0; it < nsteps; ++it) {
                const int s = it % STAGES;
                const uint32_t ph = (it / STAGES) & 1;
                if (!tc::mbar_wait_bounded(&ctl->full[s], ph, limit)) { ok = false; break; }
                tc::tc_fence_after();
                const uint32_t a_addr = tc::smem_u32(ring + s * 2 * TILE_BYTES);
                const uint32_t b_addr = diag ? a_addr : a_addr + TILE_BYTES;
#pragma unroll
                for (int kk = 0; kk < TK / 8; ++kk) {
                    const uint64_t ad = tc::sdesc_kmajor_sw128(a_addr + kk * 32);
                    const uint64_t bd = tc::sdesc_kmajor_sw128(b_addr + kk * 32);
                    tc::mma_tf32(tmem, ad, bd, idesc, (it > 0 || kk > 0) ? 1u : 0u);
                }
                tc::mma_commit(&ctl->empty[s]);
            }
            if (!ok) atomicExch(err, 1);
            tc::mma_commit(&ctl->done);
        }
    } else if (nsteps > 0) {
        // epilogue warps 2..5: TMEM lane quarter = warp % 4
        const int q = warp & 3;
        // warp-uniform decisions: tcgen05.ld needs the whole warp converged
        const bool got = __all_sync(0xffffffffu, tc::mbar_wait_bounded(&ctl->done, 0, 2 * limit));
        int e = 0;
        if (lane == 0) e = *(volatile int*)err;
        e = __shfl_sync(0xffffffffu, e, 0);
        if (!got) {
            if (lane == 0) atomicExch(err, 1);
        } else if (e == 0) {
            tc::tc_fence_after();
            // every MMA has completed (done): the operand ring is free
            float* stg = reinterpret_cast<float*>(ring) + q * 32 * 33;
            add_block_rows(tmem + ((uint32_t)(q * 32) << 16), stg, G, n, ti * TB + q * 32, tj * TB, lane);
        }
    }
    // the MMA issuer makes sure its MMAs have finished before TMEM is freed
    if (warp == 1 && lane == 0 && nsteps > 0) tc::mbar_wait_bounded(&ctl->done, 0, WAIT_LIMIT);
    __syncwarp();
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, TMEM_COLS);
    }
}

// ---------------------------------------------------------------------------
// G = X^T X of the columns of X (m x n, row-major, n contiguous): the Gram
// step of the left-to-right sweep, whose contraction runs over the rows of
// the left unfolding.  TMA brings raw 32-row x 128-column FP32 boxes; eight
// converter warps (two per scheduler) round them to TF32 and write them
// transposed into the K-major 128-byte-swizzled layout (column i of X
// becomes MMA row i), so the MMA sees the same operand form as in the row
// Gram; four of them then read the accumulator back.
// CSTG raw staging stages (a template argument: 3 or 5; five keep about
// 160 KB of loads in flight per SM, three 96 KB), COP converted operand
// stages
constexpr int COP = 2;

template <int CSTG>
struct __align__(8) ColCtl {
    uint64_t stg_full[CSTG], stg_empty[CSTG];
    uint64_t op_full[COP], op_empty[COP];
    uint64_t done;
    uint32_t tmem_base;
};

// x rounded to TF32 (10 explicit mantissa bits), to nearest with ties away
// from zero: half of the dropped 13 bits' unit added to the magnitude, then
// the dropped bits cleared (a carry moves into the exponent as it should).
// Finite inputs only matter: a NaN may come out as Inf, still non-finite.
__device__ __forceinline__ float rna_tf32(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

constexpr int CCONV = 256;  // converter threads (warps 2-9, two per scheduler)

template <int CSTG>
__global__ void __launch_bounds__(64 + CCONV, 1)
gram_cols_tf32_kernel(const __grid_constant__ CUtensorMap tmap, int n, long m, int ntiles, long kchunk_steps,
                      float* __restrict__ G, int* __restrict__ err) {
    using ColCtl = ColCtl<CSTG>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* opr = base;                           // [COP][A, B] swizzled TF32 tiles
    unsigned char* stg = opr + COP * 2 * TILE_BYTES;     // [CSTG][A raw, B raw]
    ColCtl* ctl = reinterpret_cast<ColCtl*>(stg + CSTG * 2 * TILE_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntri = ntiles * (ntiles + 1) / 2;
    const int pair = blockIdx.x % ntri;
    const long split = blockIdx.x / ntri;
    int ti = 0;
    while ((ti + 1) * (ti + 2) / 2 <= pair) ++ti;
    const int tj = pair - ti * (ti + 1) / 2;
    const bool diag = (ti == tj);
    const long ksteps_total = (m + TK - 1) / TK;
    const long ks0 = split * kchunk_steps;
    const long ks1 = min(ksteps_total, ks0 + kchunk_steps);
    const int nsteps = (int)max(0L, ks1 - ks0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < CSTG; ++s) {
            tc::mbar_init(&ctl->stg_full[s], 1);
            tc::mbar_init(&ctl->stg_empty[s], CCONV);
        }
        for (int s = 0; s < COP; ++s) {
            tc::mbar_init(&ctl->op_full[s], CCONV);
            tc::mbar_init(&ctl->op_empty[s], 1);
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
        if (lane == 0 && nsteps > 0) {
            tc::prefetch_tmap(&tmap);
            const uint32_t bytes = diag ? TILE_BYTES : 2 * TILE_BYTES;
            bool ok = true;
            int issued = 0;
            for (int it = 0; it < nsteps; ++it) {
                const int s = it % CSTG;
                if (!tc::mbar_wait_bounded(&ctl->stg_empty[s], ((it / CSTG) & 1) ^ 1, WAIT_LIMIT)) { ok = false; break; }
                unsigned char* a = stg + s * 2 * TILE_BYTES;
                tc::mbar_arrive_expect_tx(&ctl->stg_full[s], bytes);
                const int ky = (int)((ks0 + it) * TK);
                tc::tma_load_2d(a, &tmap, &ctl->stg_full[s], ti * TB, ky);
                if (!diag) tc::tma_load_2d(a + TILE_BYTES, &tmap, &ctl->stg_full[s], tj * TB, ky);
                ++issued;
            }
            if (!ok) {
                atomicExch(err, 1);
                for (int it = max(0, issued - CSTG); it < issued; ++it)
                    tc::mbar_wait_bounded(&ctl->stg_full[it % CSTG], (it / CSTG) & 1, WAIT_LIMIT);
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && nsteps > 0) {
            constexpr uint32_t idesc = tc::idesc_tf32(TB, TB);
            bool ok = true;
            for (int it = 0; it < nsteps; ++it) {
                const int o = it % COP;
                if (!tc::mbar_wait_bounded(&ctl->op_full[o], (it / COP) & 1, WAIT_LIMIT)) { ok = false; break; }
                tc::tc_fence_after();
                const uint32_t a_addr = tc::smem_u32(opr + o * 2 * TILE_BYTES);
                const uint32_t b_addr = diag ? a_addr : a_addr + TILE_BYTES;
#pragma unroll
                for (int kk = 0; kk < TK / 8; ++kk)
                    tc::mma_tf32(tmem, tc::sdesc_kmajor_sw128(a_addr + kk * 32), tc::sdesc_kmajor_sw128(b_addr + kk * 32),
                                 idesc, (it > 0 || kk > 0) ? 1u : 0u);
                tc::mma_commit(&ctl->op_empty[o]);
            }
            if (!ok) atomicExch(err, 1);
            tc::mma_commit(&ctl->done);
        }
    } else if (nsteps > 0) {
        const int t = threadIdx.x - 64;
        bool ok = true;
        for (int it = 0; it < nsteps && ok; ++it) {
            const int s = it % CSTG, o = it % COP;
            const bool g1 = tc::mbar_wait_bounded(&ctl->stg_full[s], (it / CSTG) & 1, WAIT_LIMIT);
            const bool g2 = g1 && tc::mbar_wait_bounded(&ctl->op_empty[o], ((it / COP) & 1) ^ 1, WAIT_LIMIT);
            ok = __all_sync(0xffffffffu, g1 && g2);
            if (!ok) break;
            const float* sA = reinterpret_cast<const float*>(stg + s * 2 * TILE_BYTES);  // [32 k][128 i]
            unsigned char* dA = opr + o * 2 * TILE_BYTES;
            // thread t converts half h = t / 128 of row i = t % 128 of each
            // 128 x 32 operand tile: column i of the raw box, k = 4 c .. 4 c
            // + 3 into 16-byte chunk c of the swizzled row, c = 4 h .. 4 h + 3.
            // Every load of a tile is issued before its stores (the compiler
            // cannot reorder them: both are shared memory).
            const int i = t & 127, h = t >> 7;
            const int ntile_op = diag ? 1 : 2;
            for (int u = 0; u < ntile_op; ++u) {
                const float* src = sA + u * (TILE_BYTES / 4) + i + 16 * h * TB;
                unsigned char* dst = dA + u * TILE_BYTES + i * 128;
                float r[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) r[k] = src[k * TB];
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    *reinterpret_cast<float4*>(dst + (((4 * h + c) ^ (i & 7)) << 4)) =
                        make_float4(rna_tf32(r[4 * c]), rna_tf32(r[4 * c + 1]), rna_tf32(r[4 * c + 2]),
                                    rna_tf32(r[4 * c + 3]));
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc::mbar_arrive(&ctl->op_full[o]);
            tc::mbar_arrive(&ctl->stg_empty[s]);
        }
        if (!ok && lane == 0) atomicExch(err, 1);
        if (warp < 6) {
            // epilogue on warps 2-5 (TMEM lane quarter = warp % 4)
            const int q = warp & 3;
            const bool got = __all_sync(0xffffffffu, ok && tc::mbar_wait_bounded(&ctl->done, 0, 2 * WAIT_LIMIT));
            int e = 0;
            if (lane == 0) e = *(volatile int*)err;
            e = __shfl_sync(0xffffffffu, e, 0);
            if (!got) {
                if (lane == 0) atomicExch(err, 1);
            } else if (e == 0) {
                tc::tc_fence_after();
                // every MMA has completed (done) and every staged box was
                // converted: the operand and staging smem is free
                float* stg = reinterpret_cast<float*>(base) + q * 32 * 33;
                add_block_rows(tmem + ((uint32_t)(q * 32) << 16), stg, G, n, ti * TB + q * 32, tj * TB, lane);
            }
        }
    }
    if (warp == 1 && lane == 0 && nsteps > 0) tc::mbar_wait_bounded(&ctl->done, 0, WAIT_LIMIT);
    __syncwarp();
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, TMEM_COLS);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
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

}  // namespace

bool gram_rows_tc_tf32(Ctx& c, int n, long K, const float* X, long ldx, float* G) {
    if (n <= 0 || K <= 0) return false;
    // TMA: 16-byte aligned base, row stride a multiple of 16 bytes
    if (((uintptr_t)X & 15) != 0 || (ldx * 4) % 16 != 0 || ldx < K) return false;
    if (K > (1L << 31) - 64 || n > (1 << 20)) return false;
    auto encode = get_encode();
    if (!encode) return false;
    CUtensorMap map;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)n};
    cuuint64_t strides[1] = {(cuuint64_t)ldx * 4};
    cuuint32_t box[2] = {(cuuint32_t)TK, (cuuint32_t)TB};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)X, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;

    const int ntiles = (n + TB - 1) / TB;
    const int ntri = ntiles * (ntiles + 1) / 2;
    const long ksteps = (K + TK - 1) / TK;
    long splits = std::max<long>(1, (long)c.sm_count / ntri);
    splits = std::min<long>(splits, std::max<long>(1, ksteps / 8));
    const long kchunk = (ksteps + splits - 1) / splits;
    splits = (ksteps + kchunk - 1) / kchunk;
    const long blocks = (long)ntri * splits;
    if (blocks > 2147483647L) return false;

    const size_t smem = 1024 + STAGES * 2 * TILE_BYTES + sizeof(GramSmem) + 64;
    static std::atomic<bool> attr{false};
    set_smem_once(attr, gram_tf32_kernel, (int)smem);
    int* err = c.tc_err;
    const long long limit = c.tc_wait_limit > 0 ? c.tc_wait_limit : WAIT_LIMIT;
    TT_CUDA(cudaMemsetAsync(G, 0, sizeof(float) * (size_t)n * n, c.stream));
    ProfScope ps(c, "gram_tf32_tc", (double)n * (n + 1) * (double)K, 4.0 * (double)n * K + 4.0 * n * n);
    gram_tf32_kernel<<<(unsigned)blocks, 192, smem, c.stream>>>(map, n, K, ntiles, kchunk, G, err, limit);
    TT_LAUNCHED(c);
    return true;
}

}  // namespace ttgb

namespace ttgb {

bool gram_cols_tc_tf32(Ctx& c, int n, long m, const float* X, long ldx, float* G) {
    if (n <= 0 || m <= 0) return false;
    if (((uintptr_t)X & 15) != 0 || (ldx * 4) % 16 != 0 || ldx < n) return false;
    if (m > (1L << 31) - 64 || n > (1 << 20)) return false;
    auto encode = get_encode();
    if (!encode) return false;
    CUtensorMap map;
    cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)m};
    cuuint64_t strides[1] = {(cuuint64_t)ldx * 4};
    cuuint32_t box[2] = {(cuuint32_t)TB, (cuuint32_t)TK};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)X, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    const int ntiles = (n + TB - 1) / TB;
    const int ntri = ntiles * (ntiles + 1) / 2;
    const long ksteps = (m + TK - 1) / TK;
    long splits = std::max<long>(1, (long)c.sm_count / ntri);
    splits = std::min<long>(splits, std::max<long>(1, ksteps / 8));
    const long kchunk = (ksteps + splits - 1) / splits;
    splits = (ksteps + kchunk - 1) / kchunk;
    const long blocks = (long)ntri * splits;
    if (blocks > 2147483647L) return false;
    TT_CUDA(cudaMemsetAsync(G, 0, sizeof(float) * (size_t)n * n, c.stream));
    ProfScope ps(c, "gram_tf32_tc", (double)n * (n + 1) * (double)m, 4.0 * (double)n * m + 4.0 * n * n);
    if (c.colgram_stages == 3) {
        const size_t smem = 1024 + (COP + 3) * 2 * TILE_BYTES + sizeof(ColCtl<3>) + 64;
        static std::atomic<bool> attr{false};
        set_smem_once(attr, gram_cols_tf32_kernel<3>, (int)smem);
        gram_cols_tf32_kernel<3><<<(unsigned)blocks, 64 + CCONV, smem, c.stream>>>(map, n, m, ntiles, kchunk, G, c.tc_err);
    } else {
        const size_t smem = 1024 + (COP + 5) * 2 * TILE_BYTES + sizeof(ColCtl<5>) + 64;  // 225 KB
        static std::atomic<bool> attr{false};
        set_smem_once(attr, gram_cols_tf32_kernel<5>, (int)smem);
        gram_cols_tf32_kernel<5><<<(unsigned)blocks, 64 + CCONV, smem, c.stream>>>(map, n, m, ntiles, kchunk, G, c.tc_err);
    }
    TT_LAUNCHED(c);
    return true;
}

}  // namespace ttgb
