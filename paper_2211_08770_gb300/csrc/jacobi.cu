// Truncation SVD of the left-to-right sweep of TT-round (Section 2): the
// singular values and vectors of the small R factor, by one-sided (Hestenes)
// Jacobi in FP64: plane rotations orthogonalize the rows of W = R until
// W = Sigma V^T, the rotations accumulating in U^T.
//
// FP64 arithmetic runs at 1/64 of the FP32 rate on this GPU, so one CTA
// (about 2 FP64 FMAs per clock) would need a large fraction of a second for
// a 256 x 256 factor.  The rows are therefore split into 2m blocks and m
// CTAs work at once: each round, every CTA orthogonalizes the rows of one
// pair of blocks in shared memory (pairs in round-robin order, so a sweep
// of 2m - 1 rounds meets every pair of rows), then all CTAs meet at a grid
// barrier.  The launch is cooperative (all CTAs resident); every barrier
// wait is bounded and sets the context's device error flag on expiry, after
// which all CTAs return (reported as TT_ERR_TIMEOUT by the caller).
// Small factors (p <= 32) use one CTA.
#include <cuda_runtime.h>
#include <math.h>

#include <stdlib.h>

#include <algorithm>

#include <cooperative_groups.h>

#include "internal.h"

namespace ttgb {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr long long kWaitCycles = 4000000000LL;  // about 2 s at the boost clock

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// rotation zeroing <x, y>; false when the pair is already orthogonal to tol,
// or when one of the rows is below the noise floor (squared norm <= floor2):
// such a row carries rounding noise of the larger rows, not data, and
// rotating against it only moves that noise around
__device__ __forceinline__ bool rotation(double al, double be, double ga, double tol, double floor2, double& cs,
                                         double& sn) {
    if (ga == 0.0 || fabs(ga) <= tol * sqrt(al * be) || fmin(al, be) <= floor2) return false;
    const double zeta = (be - al) / (2.0 * ga);
    const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
    cs = 1.0 / sqrt(1.0 + t * t);
    sn = cs * t;
    return true;
}

// round-robin (circle) schedule on nb = even number of players: pair k of round s
__device__ __forceinline__ void rr_pair(int nb, int s, int k, int& i, int& j) {
    if (k == 0) {
        i = s;
        j = nb - 1;
    } else {
        i = (s + k) % (nb - 1);
        j = (s - k + nb - 1) % (nb - 1);
    }
}

// grid barrier on a monotonically increasing counter; false if a wait ran
// out (the error flag is set) or another CTA reported one
__device__ bool grid_barrier(unsigned* bar, unsigned& target, int* err) {
    __shared__ int s_ok;
    __syncthreads();
    target += gridDim.x;
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        const long long t0 = clock64();
        int ok = 1;
        for (;;) {
            if (*(volatile unsigned*)bar >= target) break;
            if (*(volatile int*)err) {
                ok = 0;
                break;
            }
            if (clock64() - t0 > kWaitCycles) {
                atomicExch(err, 1);
                ok = 0;
                break;
            }
            __nanosleep(100);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// One CTA per pair of row blocks per round.  Shared memory holds the rows of
// the pair: W part (b) then U^T part (p), row stride rl = b + p.
template <int NT>
__global__ void __launch_bounds__(NT)
jacobi_coop_kernel(int p, int b, int kb, double* __restrict__ W, double* __restrict__ Ut, int max_sweeps,
                   double tol, double floor_rel, const double* __restrict__ f2, unsigned* bar, unsigned* rot,
                   int* err) {
    extern __shared__ __align__(16) double js[];
    constexpr int NW = NT / 32;
    __shared__ double red[NW][3];
    __shared__ int s_rot;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nblk = 2 * gridDim.x, rl = b + p;
    const double floor2 = floor_rel * floor_rel * (*f2);
    unsigned target = 0;
    if (tid == 0) s_rot = 0;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        for (int s = 0; s < nblk - 1; ++s) {
            int I, J;
            rr_pair(nblk, s, blockIdx.x, I, J);
            const int i0 = I * kb, ni = max(0, min(kb, p - i0));
            const int j0 = J * kb, nj = max(0, min(kb, p - j0));
            const int nr = ni + nj;
            // local row t -> global row
            auto grow = [&](int t) { return t < ni ? i0 + t : j0 + (t - ni); };
            for (int t = 0; t < nr; ++t) {
                const int g = grow(t);
                for (int e = tid; e < b; e += NT) js[(long)t * rl + e] = W[(long)g * b + e];
                for (int e = tid; e < p; e += NT) js[(long)t * rl + b + e] = Ut[(long)g * p + e];
            }
            __syncthreads();
            // cyclic sweep over the nr local rows: nloc - 1 steps of nloc / 2 pairs
            const int nloc = nr + (nr & 1);
            const int npair = nloc / 2;
            const int wpp = npair > 0 ? max(1, NW / npair) : 1;  // warps per pair
            for (int st = 0; st < nloc - 1; ++st) {
                const int pr = warp / wpp, sub = warp % wpp;
                int a = -1, c = -1;
                if (pr < npair) {
                    rr_pair(nloc, st, pr, a, c);
                    if (a >= nr || c >= nr) a = -1;
                }
                double al = 0.0, be = 0.0, ga = 0.0;
                if (a >= 0) {
                    const double* x = js + (long)a * rl;
                    const double* y = js + (long)c * rl;
                    for (int e = sub * 32 + lane; e < b; e += wpp * 32) {
                        const double u = x[e], v = y[e];
                        al = fma(u, u, al);
                        be = fma(v, v, be);
                        ga = fma(u, v, ga);
                    }
                    al = wsum(al);
                    be = wsum(be);
                    ga = wsum(ga);
                }
                if (lane == 0) {
                    red[warp][0] = al;
                    red[warp][1] = be;
                    red[warp][2] = ga;
                }
                __syncthreads();
                if (a >= 0) {
                    al = be = ga = 0.0;
                    for (int w = pr * wpp; w < pr * wpp + wpp; ++w) {
                        al += red[w][0];
                        be += red[w][1];
                        ga += red[w][2];
                    }
                    double cs, sn;
                    if (rotation(al, be, ga, tol, floor2, cs, sn)) {
                        double* x = js + (long)a * rl;
                        double* y = js + (long)c * rl;
                        for (int e = sub * 32 + lane; e < rl; e += wpp * 32) {
                            const double u = x[e], v = y[e];
                            x[e] = cs * u - sn * v;
                            y[e] = sn * u + cs * v;
                        }
                        if (lane == 0 && sub == 0) s_rot = 1;
                    }
                }
                __syncthreads();
            }
            for (int t = 0; t < nr; ++t) {
                const int g = grow(t);
                for (int e = tid; e < b; e += NT) W[(long)g * b + e] = js[(long)t * rl + e];
                for (int e = tid; e < p; e += NT) Ut[(long)g * p + e] = js[(long)t * rl + b + e];
            }
            if (s == nblk - 2 && tid == 0 && s_rot) atomicAdd(rot + sweep, 1u);
            if (!grid_barrier(bar, target, err)) return;
        }
        // every CTA reads the sweep's rotation count after the barrier: same decision
        const unsigned any = *(volatile unsigned*)(rot + sweep);
        __syncthreads();
        if (tid == 0) s_rot = 0;
        if (any == 0) break;
    }
}

// one CTA: all row pairs in round-robin order, one warp per pair, in place in global memory
__global__ void __launch_bounds__(1024)
jacobi_small_kernel(int p, int b, double* __restrict__ W, double* __restrict__ Ut, int max_sweeps, double tol,
                    double floor_rel, const double* __restrict__ f2) {
    __shared__ int s_rot;
    const double floor2 = floor_rel * floor_rel * (*f2);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int pp = p + (p & 1);
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) s_rot = 0;
        __syncthreads();
        for (int s = 0; s < pp - 1; ++s) {
            for (int k = w; k < pp / 2; k += nw) {
                int i, j;
                rr_pair(pp, s, k, i, j);
                if (i >= p || j >= p) continue;
                double* wi = W + (long)i * b;
                double* wj = W + (long)j * b;
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int t = lane; t < b; t += 32) {
                    const double x = wi[t], y = wj[t];
                    al = fma(x, x, al);
                    be = fma(y, y, be);
                    ga = fma(x, y, ga);
                }
                double cs, sn;
                if (!rotation(wsum(al), wsum(be), wsum(ga), tol, floor2, cs, sn)) continue;
                for (int q = lane; q < b; q += 32) {
                    const double x = wi[q], y = wj[q];
                    wi[q] = cs * x - sn * y;
                    wj[q] = sn * x + cs * y;
                }
                double* ui = Ut + (long)i * p;
                double* uj = Ut + (long)j * p;
                for (int q = lane; q < p; q += 32) {
                    const double x = ui[q], y = uj[q];
                    ui[q] = cs * x - sn * y;
                    uj[q] = sn * x + cs * y;
                }
                if (lane == 0) s_rot = 1;
            }
            __syncthreads();
        }
        const int r = s_rot;
        __syncthreads();
        if (!r) break;
    }
}

template <class S>
__global__ void __launch_bounds__(1024)
jacobi_prep_kernel(int p, int b, const S* __restrict__ R, double* __restrict__ W, double* __restrict__ Ut,
                   double* __restrict__ f2) {
    const long pb = (long)p * b, ppp = (long)p * p;
    double ss = 0.0;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < pb; e += (long)gridDim.x * blockDim.x) {
        const double v = (double)R[e];
        W[e] = v;
        ss = fma(v, v, ss);
    }
    ss = wsum(ss);
    if ((threadIdx.x & 31) == 0 && ss != 0.0) atomicAdd(f2, ss);
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < ppp; e += (long)gridDim.x * blockDim.x)
        Ut[e] = (e / p == e % p) ? 1.0 : 0.0;
}

// sigma_i = ||row i of W||, sorted decreasingly; SVt = sorted rows; U = sorted columns
template <class S>
__global__ void __launch_bounds__(1024)
jacobi_finish_kernel(int p, int b, const double* __restrict__ W, const double* __restrict__ Ut,
                     S* __restrict__ U, S* __restrict__ SVt, double* __restrict__ sigma) {
    extern __shared__ __align__(16) unsigned char jf_smem[];
    double* sig = reinterpret_cast<double*>(jf_smem);
    int* perm = reinterpret_cast<int*>(sig + p);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = w; i < p; i += nw) {
        double s = 0.0;
        for (int t = lane; t < b; t += 32) s = fma(W[(long)i * b + t], W[(long)i * b + t], s);
        s = wsum(s);
        if (lane == 0) sig[i] = sqrt(s);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < p; i += blockDim.x) {
        int rank = 0;
        const double si = sig[i];
        for (int j = 0; j < p; ++j) rank += (sig[j] > si) || (sig[j] == si && j < i);
        perm[rank] = i;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < p; r += blockDim.x) sigma[r] = sig[perm[r]];
    const long pb = (long)p * b;
    for (long e = threadIdx.x; e < pb; e += blockDim.x) {
        const long r = e / b, t = e % b;
        SVt[e] = (S)W[(long)perm[r] * b + t];
    }
    const long ppp = (long)p * p;
    for (long e = threadIdx.x; e < ppp; e += blockDim.x) {
        const long i = e / p, r = e % p;  // U[i][r] = Ut[perm[r]][i]
        U[e] = (S)Ut[(long)perm[r] * p + i];
    }
}

}  // namespace

template <class S>
void jacobi_svd(Ctx& c, int p, int b, const S* R, S* U, S* SVt, double* sigma, S* work, double tol,
                double floor_rel) {
    if (p <= 0) return;
    if (p > 1024 || p > b) throw_status(TT_ERR_ARG, "jacobi_svd: need p <= min(b, 1024)");
    constexpr int kMaxSweeps = 40;
    double* W = reinterpret_cast<double*>(work);
    double* Ut = W + (long)p * b;
    ProfScope ps(c, "jacobi_svd", 0.0, sizeof(S) * (2.0 * p * b + 2.0 * p * p));
    // ||R||_F^2 (noise floor), barrier counter and per-sweep rotation counts
    const size_t cbytes = 256 + sizeof(unsigned) * (1 + kMaxSweeps);
    char* cbuf = (char*)c.alloc(cbytes);
    struct Rel {
        Ctx& c;
        void* p;
        size_t b;
        ~Rel() { c.release(p, b); }
    } rel{c, cbuf, cbytes};
    TT_CUDA(cudaMemsetAsync(cbuf, 0, cbytes, c.stream));
    double* f2 = (double*)cbuf;
    unsigned* ctr = (unsigned*)(cbuf + 256);
    jacobi_prep_kernel<S><<<std::max(1, std::min(2 * c.sm_count, (int)(((long)p * b + 1023) / 1024))), 1024, 0,
                            c.stream>>>(p, b, R, W, Ut, f2);
    TT_LAUNCHED(c);
    if (p <= 32) {
        const int threads = std::min(1024, std::max(32, ((p + 1) / 2) * 32));
        jacobi_small_kernel<<<1, threads, 0, c.stream>>>(p, b, W, Ut, kMaxSweeps, tol, floor_rel, f2);
        TT_LAUNCHED(c);
    } else {
        constexpr int NT = 256;
        // blocks of kb rows, at least two per block, one CTA per block pair,
        // no more CTAs than can be resident at once
        int per_sm = 0;
        const int rl = b + p;
        // rows per block (TTGB_JACOBI_KB overrides the default of 2)
        static const int kb_env = [] {
            const char* e = getenv("TTGB_JACOBI_KB");
            return e ? std::max(1, std::min(8, atoi(e))) : 2;
        }();
        int kb = kb_env;
        auto smem_for = [&](int k) { return (size_t)2 * k * rl * sizeof(double); };
        for (;;) {
            const size_t sm = smem_for(kb);
            if (sm > 200 * 1024) throw_status(TT_ERR_ARG, "jacobi_svd: rows too long for shared memory");
            static std::atomic<bool> attr{false};
            set_smem_once(attr, jacobi_coop_kernel<NT>, 200 * 1024);
            TT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_coop_kernel<NT>, NT, sm));
            const int maxc = std::max(1, per_sm) * c.sm_count;
            const int m = ((p + kb - 1) / kb + 1) / 2;
            if (m <= maxc) break;
            if (++kb > NT / 32) throw_status(TT_ERR_ARG, "jacobi_svd: too many rows for one cooperative grid");
        }
        const int m = ((p + kb - 1) / kb + 1) / 2;
        const size_t sm = smem_for(kb);
        int pa = p, ba = b, kba = kb, ms = kMaxSweeps;
        double tl = tol, fr = floor_rel;
        unsigned* bar = ctr;
        unsigned* rot = ctr + 1;
        int* err = c.tc_err;
        void* args[] = {&pa, &ba, &kba, &W, &Ut, &ms, &tl, &fr, &f2, &bar, &rot, &err};
        TT_CUDA(cudaLaunchCooperativeKernel((const void*)jacobi_coop_kernel<NT>, dim3(m), dim3(NT), args, sm,
                                            c.stream));
        TT_LAUNCHED(c);
        if (c.prof) {  // diagnostics: sweeps run = rounds with rotations + the final check
            unsigned h[kMaxSweeps];
            TT_CUDA(cudaMemcpyAsync(h, rot, sizeof(h), cudaMemcpyDeviceToHost, c.stream));
            c.sync();
            int sw = 0;
            while (sw < kMaxSweeps && h[sw]) ++sw;
            c.stats.svd_sweeps += std::min(sw + 1, kMaxSweeps);
        }
    }
    const size_t smem = (size_t)p * (sizeof(double) + sizeof(int));
    jacobi_finish_kernel<S><<<1, 1024, smem, c.stream>>>(p, b, W, Ut, U, SVt, sigma);
    TT_LAUNCHED(c);
}

template void jacobi_svd<double>(Ctx&, int, int, const double*, double*, double*, double*, double*, double,
                                 double);
template void jacobi_svd<float>(Ctx&, int, int, const float*, float*, float*, double*, float*, double, double);


// ---------------------------------------------------------------------------
// FP32 column Jacobi for data stored in FP32 (TT_MIXED_TF32 / TT_FP32).
//
// The columns of R are orthogonalized (Hestenes: R V = U Sigma) without
// accumulating V: the converged columns are sigma_i u_i, which is all the
// truncation needs (the caller re-orthonormalizes the kept u_i and forms the
// next core's factor as U^T R, an exact orthogonal projection, so the
// truncation error is exactly the discarded part).  The rows handled here are
// the columns of R (rows of W = R^T, nr rows of length len).
//
// R is FP32 data (relative rounding 2^-24), so FP32 rotations suffice; they
// run at 64x the FP64 rate.  A thread-block cluster of C CTAs keeps all rows
// in shared memory as 2C blocks of kb rows, two per CTA.  Each round a CTA
// orthogonalizes its two blocks against each other (kb steps of kb disjoint
// pairs, one warp per pair), the first round of a sweep also within each
// block, then the blocks move to the next CTA of the circle schedule (every
// block pair meets once in 2C - 1 rounds) through distributed shared memory.
// Cluster barriers are hardware barriers: no spin-waits.
namespace {

namespace cg = cooperative_groups;

constexpr int J32_NT = 512;
constexpr int J32_MAXC = 8;

struct J32Pair {
    float* x;
    float* y;
};

// one warp: rotate rows x, y (length len) if not orthogonal to tol; true if rotated
__device__ __forceinline__ bool j32_rotate(float* x, float* y, int len, float tol, float floor2) {
    const int lane = threadIdx.x & 31;
    float al = 0.f, be = 0.f, ga = 0.f;
    for (int e = lane; e < len; e += 32) {
        const float u = x[e], v = y[e];
        al = fmaf(u, u, al);
        be = fmaf(v, v, be);
        ga = fmaf(u, v, ga);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        al += __shfl_xor_sync(FULL, al, o);
        be += __shfl_xor_sync(FULL, be, o);
        ga += __shfl_xor_sync(FULL, ga, o);
    }
    if (ga == 0.f || fabsf(ga) <= tol * sqrtf(al * be) || fminf(al, be) <= floor2) return false;
    const float zeta = (be - al) / (2.f * ga);
    const float t = fabsf(zeta) > 1e15f ? 0.5f / zeta
                                         : copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
    const float cs = rsqrtf(1.f + t * t), sn = cs * t;
    for (int e = lane; e < len; e += 32) {
        const float u = x[e], v = y[e];
        x[e] = cs * u - sn * v;
        y[e] = sn * u + cs * v;
    }
    return true;
}

__global__ void __launch_bounds__(J32_NT)
jac32_kernel(int nr, int len, int kb, float* __restrict__ W, int max_sweeps, float tol, float floor_rel,
             int* __restrict__ sweeps_out) {
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int me = (int)cl.block_rank();
    extern __shared__ __align__(16) float js32[];
    __shared__ int s_rot;
    __shared__ double s_f2;
    __shared__ int ids[2][J32_MAXC];  // block ids at the top / bottom of each CTA
    const int tid = threadIdx.x, warp = tid >> 5, NW = J32_NT / 32;
    const long bl = (long)kb * len;
    float* A0 = js32;
    float* A1 = js32 + bl;
    float* B0 = js32 + 2 * bl;
    float* B1 = js32 + 3 * bl;
    auto rows_of = [&](int blk) { return max(0, min(kb, nr - blk * kb)); };
    if (tid < C) {
        ids[0][tid] = 2 * tid;
        ids[1][tid] = 2 * tid + 1;
    }
    __syncthreads();
    // load this CTA's two blocks; missing rows are zero
    {
        const int bt = ids[0][me], bb = ids[1][me];
        for (long e = tid; e < 2 * bl; e += J32_NT) {
            const int s = (int)(e / bl);
            const long off = e % bl;
            const int blk = s == 0 ? bt : bb;
            const int r = (int)(off / len);
            float v = 0.f;
            if (r < rows_of(blk)) v = W[(long)(blk * kb + r) * len + off % len];
            js32[e] = v;
        }
    }
    // ||W||_F^2 over the cluster (noise floor)
    {
        double ss = 0.0;
        for (long e = tid; e < 2 * bl; e += J32_NT) ss += (double)js32[e] * js32[e];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(FULL, ss, o);
        if (tid == 0) s_f2 = 0.0;
        __syncthreads();
        if ((tid & 31) == 0) atomicAdd(&s_f2, ss);
        __syncthreads();
    }
    cl.sync();
    double f2 = 0.0;
    for (int r = 0; r < C; ++r) f2 += *cl.map_shared_rank(&s_f2, r);
    const float floor2 = (float)(floor_rel * floor_rel * f2);
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        if (tid == 0) s_rot = 0;
        __syncthreads();
        for (int s = 0; s < 2 * C - 1; ++s) {
            const int n0 = rows_of(ids[0][me]), n1 = rows_of(ids[1][me]);
            bool rot = false;
            if (s == 0) {
                // within each block: round-robin over kb (padded even) rows, both blocks at once
                const int kp = kb + (kb & 1);
                for (int st = 0; st < kp - 1; ++st) {
                    for (int q = warp; q < kp; q += NW) {  // q < kp/2: block 0, else block 1
                        const int b = q < kp / 2 ? 0 : 1;
                        int i, j;
                        rr_pair(kp, st, q - b * (kp / 2), i, j);
                        const int nb = b ? n1 : n0;
                        if (i < nb && j < nb) {
                            float* base = b ? A1 : A0;
                            rot |= j32_rotate(base + (long)i * len, base + (long)j * len, len, tol, floor2);
                        }
                    }
                    __syncthreads();
                }
            }
            // between the blocks: kb steps of kb disjoint pairs (i, (i + st) mod kb)
            for (int st = 0; st < kb; ++st) {
                for (int i = warp; i < kb; i += NW) {
                    const int j = (i + st) % kb;
                    if (i < n0 && j < n1) rot |= j32_rotate(A0 + (long)i * len, A1 + (long)j * len, len, tol, floor2);
                }
                __syncthreads();
            }
            if (rot && (tid & 31) == 0) s_rot = 1;
            if (C == 1) continue;
            // circle move: top of 0 stays, bottom of 0 -> top of 1, top of k -> top of k+1,
            // top of C-1 -> bottom of C-1, bottom of k+1 -> bottom of k
            cl.sync();
            {
                const int srcT = me == 0 ? 0 : (me == 1 ? 0 : me - 1);
                const int slotT = me == 0 ? 0 : (me == 1 ? 1 : 0);
                const int srcB = me == C - 1 ? C - 1 : me + 1;
                const int slotB = me == C - 1 ? 0 : 1;
                const float* rT = cl.map_shared_rank(js32 + slotT * bl, srcT);
                const float* rB = cl.map_shared_rank(js32 + slotB * bl, srcB);
                const float4* rT4 = reinterpret_cast<const float4*>(rT);
                const float4* rB4 = reinterpret_cast<const float4*>(rB);
                float4* dT = reinterpret_cast<float4*>(B0);
                float4* dB = reinterpret_cast<float4*>(B1);
                for (long e = tid; e < bl / 4; e += J32_NT) {
                    dT[e] = rT4[e];
                    dB[e] = rB4[e];
                }
            }
            cl.sync();
            {
                // new arrangement (all CTAs apply the same update)
                __shared__ int nid[2][J32_MAXC];
                if (tid < C) {
                    const int k = tid;
                    nid[0][k] = k == 0 ? ids[0][0] : (k == 1 ? ids[1][0] : ids[0][k - 1]);
                    nid[1][k] = k == C - 1 ? ids[0][C - 1] : ids[1][k + 1];
                }
                __syncthreads();
                if (tid < C) {
                    ids[0][tid] = nid[0][tid];
                    ids[1][tid] = nid[1][tid];
                }
                for (long e = tid; e < bl / 4; e += J32_NT) {
                    reinterpret_cast<float4*>(A0)[e] = reinterpret_cast<const float4*>(B0)[e];
                    reinterpret_cast<float4*>(A1)[e] = reinterpret_cast<const float4*>(B1)[e];
                }
                __syncthreads();
            }
        }
        // converged when no CTA rotated in this sweep
        cl.sync();
        int any = 0;
        for (int r = 0; r < C; ++r) any |= *cl.map_shared_rank(&s_rot, r);
        cl.sync();
        if (!any) {
            ++sweep;
            break;
        }
    }
    // rows back to W
    {
        const int bt = ids[0][me], bb = ids[1][me];
        for (long e = tid; e < 2 * bl; e += J32_NT) {
            const int s = (int)(e / bl);
            const long off = e % bl;
            const int blk = s == 0 ? bt : bb;
            const int r = (int)(off / len);
            if (r < rows_of(blk)) W[(long)(blk * kb + r) * len + off % len] = js32[e];
        }
    }
    if (me == 0 && tid == 0) *sweeps_out = sweep;
}

// sigma_i = ||row i|| (FP64 accumulation), sorted decreasingly; column r of U
// (len x nr, row-major) = the r-th row by norm, normalized (zero if sigma = 0)
__global__ void __launch_bounds__(1024)
jac32_finish_kernel(int nr, int len, int ldw, const float* __restrict__ W, float* __restrict__ U,
                    double* __restrict__ sigma) {
    extern __shared__ __align__(16) unsigned char jf32_smem[];
    double* sig = reinterpret_cast<double*>(jf32_smem);
    int* perm = reinterpret_cast<int*>(sig + nr);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = w; i < nr; i += nw) {
        double s = 0.0;
        for (int t = lane; t < len; t += 32) s = fma((double)W[(long)i * ldw + t], (double)W[(long)i * ldw + t], s);
        s = wsum(s);
        if (lane == 0) sig[i] = sqrt(s);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nr; i += blockDim.x) {
        int rank = 0;
        const double si = sig[i];
        for (int j = 0; j < nr; ++j) rank += (sig[j] > si) || (sig[j] == si && j < i);
        perm[rank] = i;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < nr; r += blockDim.x) sigma[r] = sig[perm[r]];
    const long tot = (long)len * nr;
    for (long e = threadIdx.x; e < tot; e += blockDim.x) {
        const long t = e / nr, r = e % nr;
        const int i = perm[r];
        const double s = sig[i];
        U[e] = s > 0.0 ? (float)((double)W[(long)i * ldw + t] / s) : 0.f;
    }
}

}  // namespace

bool jacobi_cols_f32(Ctx& c, int nr, int len, const float* Wsrc, long ld_src, float* Wwork, float* U,
                     double* sigma, double tol, double floor_rel) {
    if (nr <= 0 || len <= 0) return true;
    const int len4 = (len + 3) & ~3;  // rows padded with zeros to 16 bytes for the block moves
    // kb rows per block, C <= 8 CTAs with 4 block slots each in shared memory
    const int kmax = (int)((200 * 1024) / (16L * len4));
    if (kmax < 1) return false;
    int kb = std::max(1, (nr + 2 * J32_MAXC - 1) / (2 * J32_MAXC));
    kb = std::max(kb, std::min(4, (nr + 1) / 2));
    if (kb > kmax) return false;
    int C = (nr + 2 * kb - 1) / (2 * kb);
    C = std::max(1, std::min(C, J32_MAXC));
    if (2L * C * kb < nr) return false;
    const size_t smem = 16ul * kb * len4;
    static std::atomic<bool> attr{false};
    set_smem_once(attr, jac32_kernel, 200 * 1024);
    ProfScope ps(c, "jacobi_svd", 0.0, 4.0 * (2.0 * nr * len + (double)len * nr));
    if (len4 != len) TT_CUDA(cudaMemsetAsync(Wwork, 0, sizeof(float) * (size_t)nr * len4, c.stream));
    TT_CUDA(cudaMemcpy2DAsync(Wwork, len4 * sizeof(float), Wsrc, ld_src * sizeof(float), len * sizeof(float), nr,
                              cudaMemcpyDeviceToDevice, c.stream));
    int* sw = (int*)c.alloc(sizeof(int));
    struct Rel {
        Ctx& c;
        void* p;
        ~Rel() { c.release(p, sizeof(int)); }
    } rel{c, sw};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(J32_NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c.stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    TT_CUDA(cudaLaunchKernelEx(&cfg, jac32_kernel, nr, len4, kb, Wwork, 30, (float)tol, (float)floor_rel, sw));
    TT_LAUNCHED(c);
    const size_t fsm = (size_t)nr * (sizeof(double) + sizeof(int));
    jac32_finish_kernel<<<1, 1024, fsm, c.stream>>>(nr, len, len4, Wwork, U, sigma);
    TT_LAUNCHED(c);
    if (c.prof) {
        int h = 0;
        TT_CUDA(cudaMemcpyAsync(&h, sw, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
        c.sync();
        c.stats.svd_sweeps += h;
    }
    return true;
}

}  // namespace ttgb
