// Cholesky factorization with rank drop and explicit inverse of the factor:
// G + s I = L L^T, T = L^{-1}, the small r x r step of Cholesky QR in both
// sweeps of TT-round (Section 2; the Cholesky QR reading of the
// orthogonalization step).
//
// Order n <= 256 (FP32) or 160 (FP64): one CTA holds the whole lower
// triangle in shared memory as 32 x 32 tiles and reads global memory only to
// load G (L and T leave by plain stores as their tiles become final), so no
// step waits on L2 latency:
//  - right-looking Cholesky by 32-column panels: warp 0 factors and inverts
//    the diagonal tile in registers (one out-of-line, unrolled function);
//    the tiles below are multiplied by the transposed tile inverse; the
//    trailing update is spread over the warps, with warp 0 updating and
//    factoring the next diagonal tile first (lookahead), so the serial chain
//    of diagonal factorizations overlaps the bulk of the flops; finished
//    block columns of L are stored while the next ones are computed;
//  - the inverse by block rows in place of the stored rows of L, interleaved
//    with the panels: row p is T_pJ = -T_pp sum_K L_pK T_KJ, formed by the
//    warps the trailing update leaves idle, so only the last row's chain of
//    tile products follows the factorization;
//  - the status (dropped pivots, non-finite pivots, smallest pivot ratio) is
//    formed once at the end from the stored pivots, off the diagonal chain.
// (Solving the panel by forward substitution instead, with the diagonal
// inverses formed later in parallel, measured slower: the substitution's
// dependent chain per row outweighs the shorter diagonal step.)
// Tiles are stored without padding with a 16-byte-chunk XOR swizzle, so a
// lane reads its own tile row with 16-byte loads and every warp reads the
// shared operand row by 16-byte broadcasts; each 32 x 32 x 32 tile product
// is one warp, lane r owning output row r in registers.
//
// Larger orders are factored blockwise (block size NB <= the one-CTA limit)
// with the same kernel on diagonal blocks and the CUDA-core GEMM for the
// panels, trailing updates and off-diagonal inverse blocks, which spreads
// the O(n^3) work over the GPU.  NB is a fixed function of the precision
// and the order, taken from timings of every candidate on a GB300, so the
// arithmetic (and every result) is the same from run to run; it can be
// fixed per context instead.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "internal.h"

namespace ttgb {

namespace {

constexpr unsigned FULL = 0xffffffffu;

template <class C>
struct TileT;
template <>
struct TileT<float> {
    using V = float4;
    static constexpr int W = 4;     // elements per 16-byte chunk
    static constexpr int NCH = 8;   // chunks per 32-element row
    static constexpr int PMAX = 8;  // n <= 256
    __device__ __forceinline__ static void fma(float a, const float4 v, float* acc) {
        acc[0] = fmaf(a, v.x, acc[0]);
        acc[1] = fmaf(a, v.y, acc[1]);
        acc[2] = fmaf(a, v.z, acc[2]);
        acc[3] = fmaf(a, v.w, acc[3]);
    }
    __device__ __forceinline__ static void unpack(const float4 v, float* x) {
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    }
    __device__ __forceinline__ static float4 pack(const float* x) { return make_float4(x[0], x[1], x[2], x[3]); }
    __device__ __forceinline__ static float rsqrt(float x) { return rsqrtf(x); }
};
template <>
struct TileT<double> {
    using V = double2;
    static constexpr int W = 2;
    static constexpr int NCH = 16;
    static constexpr int PMAX = 5;  // n <= 160
    __device__ __forceinline__ static void fma(double a, const double2 v, double* acc) {
        acc[0] = ::fma(a, v.x, acc[0]);
        acc[1] = ::fma(a, v.y, acc[1]);
    }
    __device__ __forceinline__ static void unpack(const double2 v, double* x) {
        x[0] = v.x; x[1] = v.y;
    }
    __device__ __forceinline__ static double2 pack(const double* x) { return make_double2(x[0], x[1]); }
    __device__ __forceinline__ static double rsqrt(double x) { return 1.0 / sqrt(x); }
};

// element (r, c) of a swizzled 32 x 32 tile: chunk c / W of row r sits in
// slot (c / W) ^ (r mod NCH)
template <class C>
__device__ __forceinline__ int tix(int r, int c) {
    using TT = TileT<C>;
    return r * 32 + ((((c / TT::W) ^ (r & (TT::NCH - 1)))) * TT::W) + (c % TT::W);
}

// lane-owned row r of a tile <-> 32 registers
template <class C>
__device__ __forceinline__ void load_row(C (&x)[32], const C* tile, int r) {
    using TT = TileT<C>;
    const typename TT::V* p = reinterpret_cast<const typename TT::V*>(tile + r * 32);
#pragma unroll
    for (int j = 0; j < TT::NCH; ++j) TT::unpack(p[j ^ (r & (TT::NCH - 1))], x + j * TT::W);
}
template <class C>
__device__ __forceinline__ void store_row(C* tile, int r, const C (&x)[32]) {
    using TT = TileT<C>;
    typename TT::V* p = reinterpret_cast<typename TT::V*>(tile + r * 32);
#pragma unroll
    for (int j = 0; j < TT::NCH; ++j) p[j ^ (r & (TT::NCH - 1))] = TT::pack(x + j * TT::W);
}
// lane r's row x stored as column r of the tile (element (k, r) = x[k])
template <class C>
__device__ __forceinline__ void store_col(C* tile, int r, const C (&x)[32]) {
#pragma unroll
    for (int k = 0; k < 32; ++k) tile[tix<C>(k, r)] = x[k];
}

// acc[c] += sum_k a[k] B(k, c): B read by broadcast rows
template <class C>
__device__ __forceinline__ void tile_fma(C (&acc)[32], const C (&a)[32], const C* B) {
    using TT = TileT<C>;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const typename TT::V* row = reinterpret_cast<const typename TT::V*>(B + k * 32);
#pragma unroll
        for (int j = 0; j < TT::NCH; ++j) TT::fma(a[k], row[j ^ (k & (TT::NCH - 1))], acc + j * TT::W);
    }
}
// FP32: packed FP32x2 FMAs (a[k] duplicated once per k), the same rounding
// as fmaf on each element with half the issue slots
template <>
__device__ __forceinline__ void tile_fma<float>(float (&acc)[32], const float (&a)[32], const float* B) {
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const float4* row = reinterpret_cast<const float4*>(B + k * 32);
        unsigned long long ap;
        asm("mov.b64 %0, {%1, %1};" : "=l"(ap) : "f"(a[k]));
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float4 v = row[j ^ (k & 7)];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                unsigned long long cc, bp;
                asm("mov.b64 %0, {%1, %2};" : "=l"(cc) : "f"(acc[4 * j + 2 * h]), "f"(acc[4 * j + 2 * h + 1]));
                asm("mov.b64 %0, {%1, %2};" : "=l"(bp) : "f"(h ? v.z : v.x), "f"(h ? v.w : v.y));
                asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(cc) : "l"(ap), "l"(bp));
                asm("mov.b64 {%0, %1}, %2;" : "=f"(acc[4 * j + 2 * h]), "=f"(acc[4 * j + 2 * h + 1]) : "l"(cc));
            }
        }
    }
}

// columns [16 h, 16 h + 16) of the product only: acc[c] += sum_k a[k] B(k, 16 h + c)
// (two warps share one output tile; the same per-element rounding as tile_fma)
template <class C>
__device__ __forceinline__ void tile_fma_half(C (&acc)[16], const C (&a)[32], const C* B, int h) {
    using TT = TileT<C>;
    constexpr int HC = TT::NCH / 2;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const typename TT::V* row = reinterpret_cast<const typename TT::V*>(B + k * 32);
#pragma unroll
        for (int j = 0; j < HC; ++j) TT::fma(a[k], row[(h * HC + j) ^ (k & (TT::NCH - 1))], acc + j * TT::W);
    }
}
template <>
__device__ __forceinline__ void tile_fma_half<float>(float (&acc)[16], const float (&a)[32], const float* B, int h) {
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const float4* row = reinterpret_cast<const float4*>(B + k * 32);
        unsigned long long ap;
        asm("mov.b64 %0, {%1, %1};" : "=l"(ap) : "f"(a[k]));
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float4 v = row[(4 * h + j) ^ (k & 7)];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                unsigned long long cc, bp;
                asm("mov.b64 %0, {%1, %2};" : "=l"(cc) : "f"(acc[4 * j + 2 * e]), "f"(acc[4 * j + 2 * e + 1]));
                asm("mov.b64 %0, {%1, %2};" : "=l"(bp) : "f"(e ? v.z : v.x), "f"(e ? v.w : v.y));
                asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(cc) : "l"(ap), "l"(bp));
                asm("mov.b64 {%0, %1}, %2;" : "=f"(acc[4 * j + 2 * e]), "=f"(acc[4 * j + 2 * e + 1]) : "l"(cc));
            }
        }
    }
}
__device__ __forceinline__ int tri(int I, int J) { return I * (I + 1) / 2 + J; }  // slot of lower tile (I, J)

// Warp 0: factor the diagonal tile q in place (rank drop below tau), write
// the transposed inverse to DiT and the inverse to TD (natural layout), and
// the pivots to pivs[32 q ..] (the status is formed from them once, at the
// end of the kernel: its FP64 ratios and reductions stay off this chain).
// Lane r holds row r in registers.  Step c: the pivot comes from lane c,
// column c is scaled, published in col[] and subtracted from the rows below
// (16-byte broadcast reads of col; entries above the diagonal are zeroed at
// their own step; broadcasting by register shuffles instead measured 30%
// slower).  Kept out of line: inlined into the kernel, the compiler
// schedules this dependent chain several times slower.
template <class C>
__device__ __noinline__ void factor_diag(int q, C* Lt, C* DiT, C* TD, C* col, C* pivs, double tau) {
    using TT = TileT<C>;
    const int lane = threadIdx.x & 31;
    C* tile = Lt + (long)tri(q, q) * 1024;
    C a[32];
    load_row<C>(a, tile, lane);
    C invs[32];
    const C tau_c = (C)tau;
    C mypiv = C(0);  // lane c keeps pivot c
    // next pivot, updated by lane c+1 from its own multiplier: the same FMA
    // the column broadcast below applies to it, formed before the broadcast
    // so the pivot chain (shuffle, rsqrt, multiply) skips the shared-memory
    // round trip
    C pnext = a[0];
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        const C piv = __shfl_sync(FULL, pnext, c);
        const bool keep = isfinite(piv) && piv > tau_c && piv > C(0);
        // reciprocal square root first: one special-function op on the
        // pivot chain in FP32 (2 ulp; Cholesky's backward error is O(n u))
        const C inv = keep ? TT::rsqrt(piv) : C(0);
        invs[c] = inv;
        if (lane == c) mypiv = piv;
        const C l = (lane > c) ? a[c] * inv : C(0);
        if (c + 1 < 32) pnext = fma(-l, l, a[c + 1]);
        a[c] = (lane == c) ? piv * inv : l;
        col[lane] = l;
        __syncwarp();
        const typename TT::V* cv = reinterpret_cast<const typename TT::V*>(col);
#pragma unroll
        for (int j = (c + 1) / TT::W; j < TT::NCH; ++j) {
            C l4[TT::W];
            TT::unpack(cv[j], l4);
#pragma unroll
            for (int e = 0; e < TT::W; ++e)
                if (j * TT::W + e > c) a[j * TT::W + e] = fma(-l, l4[e], a[j * TT::W + e]);
        }
        __syncwarp();
    }
    store_row<C>(tile, lane, a);
    pivs[q * 32 + lane] = mypiv;
    __syncwarp();
    // inverse: lane c solves column c, x_i = (delta_ic - sum_{k<i} L_ik x_k) / L_ii,
    // L_ik read back from the tile by broadcast loads, two partial sums
    // (loading row i in 16-byte chunks instead measured 3-4x slower)
    C x[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        C s0 = (i == lane) ? C(1) : C(0), s1 = C(0);
#pragma unroll
        for (int k = 0; k < i; ++k) {
            if (k & 1) s1 = fma(-tile[tix<C>(i, k)], x[k], s1);
            else s0 = fma(-tile[tix<C>(i, k)], x[k], s0);
        }
        x[i] = (s0 + s1) * invs[i];
    }
    store_row<C>(DiT, lane, x);                // DiT row c = column c of T_qq
    store_col<C>(TD + (long)q * 1024, lane, x);  // TD natural: (i, c) = x_i of lane c
    __syncwarp();
}

// row r of tile (I, J) of an n x n matrix from a lane's registers, columns
// [16 h0, 16 h0 + 16 NH) (x holds them from x[0]), clipped to n
template <class S, class C, int NH>
__device__ __forceinline__ void gstore_row(S* out, long ld, int n, int I, int J, int r, const C* x, int h0) {
    const int gi = I * 32 + r, gj0 = J * 32 + 16 * h0;
    if (gi >= n) return;
    S* o = out + (long)gi * ld + gj0;
    using TT = TileT<C>;
    if (sizeof(S) == sizeof(C) && gj0 + 16 * NH <= n && ((ld % TT::W) == 0) && ((((uintptr_t)o) & 15) == 0)) {
#pragma unroll
        for (int j = 0; j < 16 * NH / TT::W; ++j)
            *reinterpret_cast<typename TT::V*>(o + j * TT::W) = TT::pack(x + j * TT::W);
    } else {
#pragma unroll
        for (int c = 0; c < 16 * NH; ++c)
            if (gj0 + c < n) o[c] = (S)x[c];
    }
}

// zeros of the n x n lower-triangular inverse above its diagonal tiles (the
// diagonal tiles are stored whole), one warp per row, by warps [w0, w0 + nw)
template <class S>
__device__ void zero_upper(int n, S* out, long ld, int w, int nw, int lane) {
    for (int gi = w; gi < n; gi += nw) {
        S* o = out + (long)gi * ld;
        for (int gj = (gi / 32 + 1) * 32 + lane; gj < n; gj += 32) o[gj] = S(0);
    }
}

// block column p of the n x n factor from the tiles (zeros above the
// diagonal), 16-byte chunks, by threads [0, nthr) of the CTA (t0 = own index)
template <class S, class C>
__device__ void store_lcol(int n, int P, int p, const C* Lt, S* out, long ld, int t0, int nthr) {
    using TT = TileT<C>;
    const bool vec = ((ld % TT::W) == 0) && ((((uintptr_t)out) & 15) == 0);
    const int nitem = P * 32 * TT::NCH;
    for (int e = t0; e < nitem; e += nthr) {
        const int I = e / (32 * TT::NCH), r = (e / TT::NCH) & 31, ch = e % TT::NCH;
        const int gi = I * 32 + r, gj0 = p * 32 + ch * TT::W;
        if (gi >= n || gj0 >= n) continue;
        C v[TT::W];
        if (I >= p) {
            TT::unpack(*reinterpret_cast<const typename TT::V*>(Lt + (long)tri(I, p) * 1024 + r * 32 +
                                                                  ((ch ^ (r & (TT::NCH - 1))) * TT::W)),
                       v);
            if (I == p) {
#pragma unroll
                for (int w = 0; w < TT::W; ++w)
                    if (ch * TT::W + w > r) v[w] = C(0);
            }
        } else {
#pragma unroll
            for (int w = 0; w < TT::W; ++w) v[w] = C(0);
        }
        if (vec && gj0 + TT::W <= n) {
            *reinterpret_cast<typename TT::V*>(out + (long)gi * ld + gj0) = TT::pack(v);
        } else {
#pragma unroll
            for (int w = 0; w < TT::W; ++w)
                if (gj0 + w < n) out[(long)gi * ld + gj0 + w] = (S)v[w];
        }
    }
}

// Arguments of one factorization.  Standalone (ext == nullptr): the shift is
// shift_rel trace(G), the drop threshold drop_rel (max_j G_jj + shift); both
// applied here and the status written.  Block of a larger factorization
// (ext != nullptr): G already carries the shift, ext[0] = shift and ext[1]
// = drop threshold, od_src is the original diagonal of the whole matrix at
// this block, and the status is merged atomically.
template <class S>
struct TileArgs {
    int n;
    const S* G;
    long ldg;
    S* L;
    long ldl;
    S* T;
    long ldt;
    const S* od_src;  // original diagonal: od_src[i * od_stride]
    long od_stride;
    double shift_rel, drop_rel;
    const double* ext;
    CholStatus* st;
};

// T_pJ = sum_{K=J}^{p-1} M_pK T_KJ for J < p: M_pK = -T_pp L_pK in tile
// slot (p, K), T_KJ in slot (K, J), T_JJ in TD; one warp, lane r's row r in
// acc (a block row of the forward substitution L T = I)
template <class C>
__device__ __forceinline__ void inv_row_tile(C (&acc)[32], int p, int J, const C* Lt, const C* TD, int lane) {
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = C(0);
    for (int K = J; K < p; ++K) {
        C x[32];
        load_row<C>(x, Lt + (long)tri(p, K) * 1024, lane);
        tile_fma<C>(acc, x, K == J ? TD + (long)J * 1024 : Lt + (long)tri(K, J) * 1024);
    }
}

// columns [16 h, 16 h + 16) of the same tile
template <class C>
__device__ __forceinline__ void inv_row_half(C (&acc)[16], int p, int J, int h, const C* Lt, const C* TD, int lane) {
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = C(0);
    for (int K = J; K < p; ++K) {
        C x[32];
        load_row<C>(x, Lt + (long)tri(p, K) * 1024, lane);
        tile_fma_half<C>(acc, x, K == J ? TD + (long)J * 1024 : Lt + (long)tri(K, J) * 1024, h);
    }
}

__device__ __forceinline__ void atomic_min_nonneg(double* addr, double v) {
    // non-negative doubles order like their bit patterns
    atomicMin(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

template <class S, class C, int NT>
__global__ void __launch_bounds__(NT) chol_tile_kernel(TileArgs<S> A) {
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) unsigned char ct_smem[];
    __shared__ double od[TileT<C>::PMAX * 32];
    __shared__ double red[2 * NW];
    __shared__ __align__(16) C colbuf[32];
    __shared__ C pivs[TileT<C>::PMAX * 32];
    const int n = A.n;
    const int P = (n + 31) / 32;
    const int ntile = P * (P + 1) / 2;
    C* Lt = reinterpret_cast<C*>(ct_smem);   // ntile tiles
    C* PT = Lt + (long)ntile * 1024;         // P - 1 tiles (panel transposed / trtri rows)
    C* DiT = PT + (long)(P - 1) * 1024;      // 1 tile
    C* TD = DiT + 1024;                      // P tiles (diagonal inverses)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // ---- shift and drop threshold
    double shift, tau, addshift, tr = 0.0, mx = 0.0;
    if (A.ext) {
        shift = A.ext[0];
        tau = A.ext[1];
        addshift = 0.0;
    } else {
        for (int i = tid; i < n; i += NT) {
            const double g = (double)A.G[(long)i * A.ldg + i];
            tr += g;
            mx = fmax(mx, g);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            tr += __shfl_xor_sync(FULL, tr, o);
            mx = fmax(mx, __shfl_xor_sync(FULL, mx, o));
        }
        if (lane == 0) {
            red[warp] = tr;
            red[NW + warp] = mx;
        }
        __syncthreads();
        tr = 0.0;
        mx = 0.0;
        for (int w = 0; w < NW; ++w) {
            tr += red[w];
            mx = fmax(mx, red[NW + w]);
        }
        shift = A.shift_rel * tr;
        tau = A.drop_rel * (mx + shift);
        addshift = shift;
    }
    for (int i = tid; i < P * 32; i += NT) od[i] = (i < n) ? (double)A.od_src[(long)i * A.od_stride] + shift : 1.0;

    // ---- load the lower tiles of G (+ shift on the diagonal); padding = identity.
    // One 16-byte chunk (W consecutive columns of a tile row) per item: the
    // in-range chunks as asynchronous copies (all in flight at once), the
    // rest by plain loads; then the diagonal tiles are fixed up (zeros above
    // the diagonal, shift on it).
    {
        using TT = TileT<C>;
        __shared__ unsigned char s_I[64], s_J[64];
        if (tid < ntile) {
            int I = 0;
            while ((I + 1) * (I + 2) / 2 <= tid) ++I;
            s_I[tid] = (unsigned char)I;
            s_J[tid] = (unsigned char)(tid - I * (I + 1) / 2);
        }
        __syncthreads();
        const bool vec = ((A.ldg % TT::W) == 0) && ((((uintptr_t)A.G) & 15) == 0);
        const int nitem = ntile * 32 * TT::NCH;
        for (int e = tid; e < nitem; e += NT) {
            const int slot = e / (32 * TT::NCH), r = (e / TT::NCH) & 31, ch = e % TT::NCH;
            const int I = s_I[slot], J = s_J[slot];
            const int gi = I * 32 + r, gj0 = J * 32 + ch * TT::W;
            C* dst = Lt + (long)slot * 1024 + r * 32 + ((ch ^ (r & (TT::NCH - 1))) * TT::W);
            if (vec && gi < n && gj0 + TT::W <= n) {
                const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa),
                             "l"(A.G + (long)gi * A.ldg + gj0));
            } else {
                C v[TT::W];
#pragma unroll
                for (int w = 0; w < TT::W; ++w) {
                    const int gj = gj0 + w;
                    v[w] = (gi < n && gj < n) ? (C)A.G[(long)gi * A.ldg + gj] : (gi == gj ? C(1) : C(0));
                }
                *reinterpret_cast<typename TT::V*>(dst) = TT::pack(v);
            }
        }
        asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
        for (int e = tid; e < P * 1024; e += NT) {
            const int J = e >> 10, r = (e >> 5) & 31, cc = e & 31;
            const int gi = J * 32 + r;
            C* t = Lt + (long)tri(J, J) * 1024 + tix<C>(r, cc);
            if (cc > r) *t = C(0);
            else if (cc == r && gi < n) *t = (C)((double)*t + addshift);
        }
    }
    __syncthreads();

    // ---- Cholesky, right-looking by panels, diagonal factor one panel ahead,
    // and the inverse T = L^{-1} one block row per panel, in place of the
    // rows of L that are final and stored: row p from
    //   M_pK = -T_pp L_pK  (K < p, over L_pK, during the panel solve), then
    //   T_pJ = sum_{K=J}^{p-1} M_pK T_KJ  (J < p, during the trailing update),
    // the tile T_pJ by one warp, held in registers across the barrier that
    // ends the panel and stored at the start of the next one (the in-place
    // reads of row p are complete by then).  The serial chain left after the
    // last panel is P - 1 half-tile products.
    // worker warps: those that do not share warp 0's scheduler (warp mod 4
    // != 0), so that the serial chain of diagonal factorizations issues
    // without contention while the workers update the trailing matrix
    constexpr int NWK = NW - NW / 4;
    static_assert(TileT<C>::PMAX - 1 <= NWK, "one inverse tile per worker and a worker for the trailing update");
    C held[32];
    int held_slot = -1, held_J = 0;
    // T leaves the CTA as its tiles become final: the zeros above the
    // diagonal tiles now, T_pp and the tiles of row p - 1 at the start of
    // panel p, the last row at the end
    if (warp == 0) factor_diag<C>(0, Lt, DiT, TD, colbuf, pivs, tau);
    else zero_upper<S>(n, A.T, A.ldt, warp - 1, NW - 1, lane);
    __syncthreads();
    for (int p = 0; p < P; ++p) {
        const int R = P - 1 - p;
        if (held_slot >= 0) {
            store_row<C>(Lt + (long)held_slot * 1024, lane, held);
            gstore_row<S, C, 2>(A.T, A.ldt, n, p - 1, held_J, lane, held, 0);
            held_slot = -1;
        }
        if (warp == R) {  // T_pp (a warp the panel solve and M_pK leave free)
            C x[32];
            load_row<C>(x, TD + (long)p * 1024, lane);
            gstore_row<S, C, 2>(A.T, A.ldt, n, p, p, lane, x, 0);
        }
        // panel solve: L_Ip = A_Ip T_pp^T, natural copy in place and transposed copy in PT
        for (int I = p + 1 + warp; I < P; I += NW) {
            C* tile = Lt + (long)tri(I, p) * 1024;
            C a[32], acc[32];
            load_row<C>(a, tile, lane);
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[j] = C(0);
            tile_fma<C>(acc, a, DiT);
            store_row<C>(tile, lane, acc);
            store_col<C>(PT + (long)(I - p - 1) * 1024, lane, acc);
        }
        // M_pK = -T_pp L_pK, in place (the warps from the top)
        {
            const int K = NW - 1 - warp;
            if (K < p) {
                C* tile = Lt + (long)tri(p, K) * 1024;
                C a[32], acc[32];
                load_row<C>(a, TD + (long)p * 1024, lane);
#pragma unroll
                for (int k = 0; k < 32; ++k) a[k] = -a[k];
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[j] = C(0);
                tile_fma<C>(acc, a, tile);
                __syncwarp();
                store_row<C>(tile, lane, acc);
            }
        }
        __syncthreads();
        if (R == 0) break;
        // trailing update A_IK -= L_Ip L_Kp^T for p < K <= I: warp 0 first
        // takes (p+1, p+1) and factors it; the workers take the trailing
        // tiles (workers 0 .. NWK-1-p) and row p of T (tile J by worker
        // NWK-1-J)
        const int ntask = R * (R + 1) / 2;
        const int wk = (warp & 3) ? warp - (warp >> 2) - 1 : -1;
        const int ntw = NWK - p;
        if (warp == 0) {
            C* tile = Lt + (long)tri(p + 1, p + 1) * 1024;
            C a[32], acc[32];
            load_row<C>(acc, tile, lane);
            load_row<C>(a, Lt + (long)tri(p + 1, p) * 1024, lane);
#pragma unroll
            for (int k = 0; k < 32; ++k) a[k] = -a[k];
            tile_fma<C>(acc, a, PT);
            store_row<C>(tile, lane, acc);
            __syncwarp();
            factor_diag<C>(p + 1, Lt, DiT, TD, colbuf, pivs, tau);
        } else if (wk >= 0 && wk < ntw) {
            // tasks 1..ntask-1 in (I, K) order over I = p+1.., K = p+1..I; task 0 is (p+1, p+1)
            for (int t = wk + 1; t < ntask; t += ntw) {
                int ii = 0;
                while ((ii + 1) * (ii + 2) / 2 <= t) ++ii;
                const int kk = t - ii * (ii + 1) / 2;
                const int I = p + 1 + ii, K = p + 1 + kk;
                C* tile = Lt + (long)tri(I, K) * 1024;
                C a[32], acc[32];
                load_row<C>(acc, tile, lane);
                load_row<C>(a, Lt + (long)tri(I, p) * 1024, lane);
#pragma unroll
                for (int k = 0; k < 32; ++k) a[k] = -a[k];
                tile_fma<C>(acc, a, PT + (long)(K - p - 1) * 1024);
                store_row<C>(tile, lane, acc);
            }
        } else if (wk >= 0) {
            const int J = NWK - 1 - wk;
            if (J < p) {
                inv_row_tile<C>(held, p, J, Lt, TD, lane);
                held_slot = tri(p, J);
                held_J = J;
            }
        }
        // block column p of L is final: the workers store it while warp 0
        // factors the next diagonal tile
        if (wk >= 0) store_lcol<S, C>(n, P, p, Lt, A.L, A.ldl, wk * 32 + lane, NWK * 32);
        __syncthreads();
    }
    // the last block row of T, straight to global memory, and the last block
    // column of L; with warps to spare, tile J by warps 2J and 2J+1, a half
    // of its columns each
    constexpr bool HALF = 2 * (TileT<C>::PMAX - 1) <= NW;
    C lrow[HALF ? 16 : 32];
    const int Jl = HALF ? warp >> 1 : warp, hl = HALF ? warp & 1 : 0;
    if (Jl < P - 1) {
        if constexpr (HALF) {
            inv_row_half<C>(lrow, P - 1, Jl, hl, Lt, TD, lane);
            gstore_row<S, C, 1>(A.T, A.ldt, n, P - 1, Jl, lane, lrow, hl);
        } else {
            inv_row_tile<C>(lrow, P - 1, Jl, Lt, TD, lane);
            gstore_row<S, C, 2>(A.T, A.ldt, n, P - 1, Jl, lane, lrow, 0);
        }
    }
    store_lcol<S, C>(n, P, P - 1, Lt, A.L, A.ldl, tid, NT);
    // status from the pivots (warp 0 wrote them): dropped (not finite, not
    // above tau, not positive) and non-finite counts, and the smallest
    // ratio of a kept pivot to its original diagonal entry
    if (warp == 0) {
        const C tau_c = (C)tau;
        int ndrop = 0, nonfin = 0;
        double minratio = 1e300;
        for (int j = lane; j < n; j += 32) {
            const C pv = pivs[j];
            const bool keep = isfinite(pv) && pv > tau_c && pv > C(0);
            nonfin |= !isfinite(pv);
            ndrop += !keep;
            if (keep) minratio = fmin(minratio, od[j] > 0.0 ? (double)pv / od[j] : 0.0);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ndrop += __shfl_xor_sync(FULL, ndrop, o);
            nonfin |= __shfl_xor_sync(FULL, nonfin, o);
            minratio = fmin(minratio, __shfl_xor_sync(FULL, minratio, o));
        }
        if (lane == 0) {
            if (A.ext) {
                if (ndrop) atomicAdd(&A.st->ndrop, ndrop);
                if (nonfin) atomicOr(&A.st->nonfinite, 1);
                atomic_min_nonneg(&A.st->min_ratio, minratio);
            } else {
                A.st->ndrop = ndrop;
                A.st->nonfinite = nonfin;
                A.st->min_ratio = minratio > 1e299 ? 0.0 : minratio;
                A.st->trace = tr;
                A.st->max_diag = mx;
            }
        }
    }
}

// Blocked driver preparation, one launch: every block reduces the diagonal
// (trace and maximum: n loads, the same in every block) for the shift
// shift_rel trace(G) and the drop threshold drop_rel (max_j G_jj + shift);
// block 0 publishes them (ext) and initialises the status; all blocks copy
// L = lower(G) + shift I (strictly upper part zero) and zero T.
template <class S>
__global__ void chol_prep_kernel(int n, const S* __restrict__ G, double shift_rel, double drop_rel,
                                 double* __restrict__ ext, CholStatus* __restrict__ st, S* __restrict__ L,
                                 S* __restrict__ T) {
    __shared__ double rt[32], rm[32], sh;
    double tr = 0.0, mx = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double g = (double)G[(long)i * n + i];
        tr += g;
        mx = fmax(mx, g);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tr += __shfl_xor_sync(FULL, tr, o);
        mx = fmax(mx, __shfl_xor_sync(FULL, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        rt[threadIdx.x >> 5] = tr;
        rm[threadIdx.x >> 5] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        tr = 0.0;
        mx = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            tr += rt[w];
            mx = fmax(mx, rm[w]);
        }
        const double shift = shift_rel * tr;
        sh = shift;
        if (blockIdx.x == 0) {
            ext[0] = shift;
            ext[1] = drop_rel * (mx + shift);
            st->ndrop = 0;
            st->nonfinite = 0;
            st->min_ratio = 1e300;
            st->trace = tr;
            st->max_diag = mx;
        }
    }
    __syncthreads();
    const double shift = sh;
    const long total = (long)n * n;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const long i = e / n, j = e % n;
        S v = S(0);
        if (j <= i) v = (i == j) ? (S)((double)G[e] + shift) : G[e];
        L[e] = v;
        T[e] = S(0);
    }
}

template <class S, class C>
constexpr int tile_nt() {
    return sizeof(C) == 4 ? 512 : 256;  // FP32: 16 warps share the tile products
}

template <class S, class C>
size_t tile_smem(int n) {
    const int P = (n + 31) / 32;
    return sizeof(C) * 1024 * (size_t)(P * (P + 1) / 2 + (P - 1) + 1 + P);
}

template <class S, class C>
void launch_tile(Ctx& c, const TileArgs<S>& a) {
    constexpr int NT = tile_nt<S, C>();
    const int nmax = TileT<C>::PMAX * 32;
    static std::atomic<bool> attr{false};
    set_smem_once(attr, chol_tile_kernel<S, C, NT>, (int)tile_smem<S, C>(nmax));
    chol_tile_kernel<S, C, NT><<<1, NT, tile_smem<S, C>(a.n), c.stream>>>(a);
    TT_LAUNCHED(c);
}

void mark_chol(Ctx& c) {
    if (!c.chol_mark) return;
    cudaEvent_t e = c.chol_mark;
    c.chol_mark = nullptr;
    TT_CUDA(cudaEventRecord(e, c.stream));
}

template <class S, class C>
void blocked(Ctx& c, int n, int nb, const S* G, S* L, S* T, double shift_rel, double drop_rel, CholStatus* st) {
    const int m = (n + nb - 1) / nb;
    const size_t wbytes = sizeof(S) * (size_t)n * nb + 2 * sizeof(double) + 256;
    char* ws = (char*)c.alloc(wbytes);
    // released on the stream of the last products that read it
    struct Rel {
        Ctx& c;
        void* p;
        size_t b;
        cudaStream_t on;
        ~Rel() {
            const cudaStream_t s0 = c.stream;
            c.stream = on;
            c.release(p, b);
            c.stream = s0;
        }
    } rel{c, ws, wbytes, c.stream};
    double* ext = (double*)ws;
    S* W = (S*)(ws + 256);
    const int cb = std::min(2 * c.sm_count, (int)(((long)n * n + 255) / 256));
    chol_prep_kernel<S><<<std::max(cb, 1), 256, 0, c.stream>>>(n, G, shift_rel, drop_rel, ext, st, L, T);
    TT_LAUNCHED(c);
    mark_chol(c);
    const long ld = n;
    for (int j = 0; j < m; ++j) {
        const int j0 = j * nb, b = std::min(nb, n - j0), j1 = j0 + b, M = n - j1;
        TileArgs<S> a{b, L + j0 * (ld + 1), ld, L + j0 * (ld + 1), ld, T + j0 * (ld + 1), ld,
                      G + j0 * (ld + 1), ld + 1, 0.0, 0.0, ext, st};
        if (M == 0 && j > 0 && c.chol_mark2) {
            // before the last tile kernel: L's columns left of this block are
            // final (the last block writes only its own columns)
            cudaEvent_t e = c.chol_mark2;
            c.chol_mark2 = nullptr;
            TT_CUDA(cudaEventRecord(e, c.stream));
            c.chol_split = j0;
        }
        launch_tile<S, C>(c, a);
        if (M == 0) break;
        // panel L_{>j,j} = A_{>j,j} T_jj^T (via W), then the trailing update
        gemm<S>(c, false, true, M, b, b, S(1), L + j1 * ld + j0, ld, T + j0 * (ld + 1), ld, S(0), W, b, 1, 0, 0, 0,
                TRI_B_UPPER);
        TT_CUDA(cudaMemcpy2DAsync(L + j1 * ld + j0, ld * sizeof(S), W, b * sizeof(S), b * sizeof(S), M,
                                  cudaMemcpyDeviceToDevice, c.stream));
        // lower triangle only (the strictly upper part of L is zeroed at the end)
        gemm<S>(c, false, true, M, M, b, S(-1), W, b, W, b, S(1), L + j1 * (ld + 1), ld, 1, 0, 0, 0, TRI_C_LOWER);
    }
    // off-diagonal inverse blocks, last block column first:
    // T_{>j,j} = -T_{>j,>j} (L_{>j,j} T_jj); on the context's tail stream
    // when one is set (L is final here: only T's readers wait for them)
    cudaStream_t saved = c.stream;
    if (c.chol_tail && m >= 2) {
        cudaEvent_t e = c.event();
        TT_CUDA(cudaEventRecord(e, c.stream));
        TT_CUDA(cudaStreamWaitEvent(c.chol_tail, e, 0));
        c.ev_pool.push_back(e);
        c.stream = c.chol_tail;
        rel.on = c.chol_tail;
    }
    struct Restore {
        Ctx& c;
        cudaStream_t s;
        ~Restore() { c.stream = s; }
    } restore{c, saved};
    for (int j = m - 2; j >= 0; --j) {
        const int j0 = j * nb, b = std::min(nb, n - j0), j1 = j0 + b, M = n - j1;
        gemm<S>(c, false, false, M, b, b, S(1), L + j1 * ld + j0, ld, T + j0 * (ld + 1), ld, S(0), W, b, 1, 0, 0, 0,
                TRI_B_LOWER);
        gemm<S>(c, false, false, M, b, M, S(-1), T + j1 * (ld + 1), ld, W, b, S(0), T + j1 * ld + j0, ld, 1, 0, 0, 0,
                TRI_A_LOWER);
    }
    // L's strictly upper part is still zero: the diagonal blocks are stored
    // with zeros above their diagonal and the trailing products write lower
    // elements only (TRI_C_LOWER)
}

// Block size per precision and order (the one-CTA kernel when it fits).
// Measured on a GB300 (microseconds, every candidate NB), fastest kept:
//   FP32: one CTA up to 256 (n = 256: 117); n = 288-320: NB 160 (145, 157);
//   n = 352-448: NB 224 (179, 206, 226); n = 512: NB 256 (270);
//   n = 640-800: NB 224 (339, 459).
//   FP64: one CTA up to 160; above, NB 128 (n = 256: 1334, 400: 2322,
//   512: 2920, 800: 5058; NB 64 was 4-10% slower).
int default_nb(int es, int n, int nmax) {
    if (n <= nmax) return n;
    if (es == 8) return 128;
    if (n <= 320) return 160;
    if (n <= 480) return 224;
    if (n <= 544) return 256;
    return 224;
}

}  // namespace


template <class S, class C>
int chol_tile_max() {
    return TileT<C>::PMAX * 32;
}

template <class S, class C>
void chol_inv_nb(Ctx& c, int n, int nb, const S* G, S* L, S* T, double shift_rel, double drop_rel, CholStatus* st) {
    const int nmax = chol_tile_max<S, C>();
    if (nb >= n && n <= nmax) {
        TileArgs<S> a{n, G, n, L, n, T, n, G, (long)n + 1, shift_rel, drop_rel, nullptr, st};
        mark_chol(c);
        launch_tile<S, C>(c, a);
    } else {
        blocked<S, C>(c, n, std::max(32, std::min(nb, nmax)), G, L, T, shift_rel, drop_rel, st);
    }
}

template <class S, class C>
void chol_inv(Ctx& c, int n, const S* G, S* L, S* T, double shift_rel, double drop_rel, CholStatus* st) {
    if (n <= 0) return;
    const int nmax = chol_tile_max<S, C>();
    ProfScope ps(c, "chol_inv", 2.0 * (double)n * n * n / 3.0, 3.0 * sizeof(S) * n * n);
    const int nb = c.chol_nb ? c.chol_nb : default_nb((int)sizeof(C), n, nmax);
    chol_inv_nb<S, C>(c, n, nb, G, L, T, shift_rel, drop_rel, st);
}

template void chol_inv<double, double>(Ctx&, int, const double*, double*, double*, double, double, CholStatus*);
template void chol_inv<float, float>(Ctx&, int, const float*, float*, float*, double, double, CholStatus*);
template void chol_inv_nb<double, double>(Ctx&, int, int, const double*, double*, double*, double, double,
                                          CholStatus*);
template void chol_inv_nb<float, float>(Ctx&, int, int, const float*, float*, float*, double, double, CholStatus*);
template int chol_tile_max<double, double>();
template int chol_tile_max<float, float>();

}  // namespace ttgb
