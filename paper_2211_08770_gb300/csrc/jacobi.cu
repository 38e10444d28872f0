// Truncation SVD of the left-to-right sweep of TT-round (Section 2.3): the
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

}  // namespace ttgb
