// Kernels and host driver of the solver.  Every step of Algorithm 1 runs in
// a kernel below; the host only sizes allocations and launches from the
// counts the kernels report (one small device-to-host read per tree level).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <cstdio>
#include <cstring>
#include <vector>

#include "mrrr.h"
#include "mrrr_entry.h"
#include "mrrr_phases.cuh"

namespace mrrr {

constexpr int kThreads = 128;

// Kernels that run one long serial recurrence per thread (bisection, RQI,
// child shifts) are bound by the latency of their FP64 chains and by the
// FP64 issue rate of each SM sub-partition, not by memory.  They launch
// one-warp CTAs so that even a few thousand items spread over all 152 SMs
// instead of piling into a few large CTAs.
constexpr int kLatThreads = 32;
// threads of the one-CTA-per-block root kernel
constexpr int kRootThreads = 256;
inline int grid_for(long long n, int threads = kThreads) { return (int)((n + threads - 1) / threads); }

// ------------------------------------------------------------------ kernels

// Low precision used for the pre-bisection under each working precision.
template <class Y> struct LowOf { typedef float T; static constexpr bool use = false; };
template <> struct LowOf<double> { typedef float T; static constexpr bool use = true; };
template <> struct LowOf<dd> { typedef double T; static constexpr bool use = true; };

// Preprocessing (Sec. 2 and Sec. 3.2, "Preprocessing"), one CTA per matrix:
// ||T||_1 by a max-reduction, scaling by the power of two that brings it to
// [1/2, 1), splitting where |e_i| <= eps_x ||T||_1, and the compact list of
// blocks by a CTA-wide scan.  Same results as prep_matrix.
template <class X>
__global__ void k_prep(MatrixDesc* mats, BlockDesc* blocks, double* wd, double* we, SolveCfg cfg) {
    constexpr int T = 256;
    __shared__ double red[T];
    __shared__ int cnt[T];
    __shared__ int bad;
    MatrixDesc& M = mats[blockIdx.x];
    const int n = M.n;
    const int tid = threadIdx.x;
    if (tid == 0) bad = 0;
    __syncthreads();
    double mx = 0.0;
    for (int i = tid; i < n; i += T) {
        double di = ld_x<X>(M.d, i);
        double sum = fabs(di);
        if (!isfinite(di)) bad = 1;
        if (i > 0) sum += fabs(ld_x<X>(M.e, i - 1));
        if (i < n - 1) {
            double ei = ld_x<X>(M.e, i);
            if (!isfinite(ei)) bad = 1;
            sum += fabs(ei);
        }
        mx = fmax(mx, sum);
    }
    red[tid] = mx;
    __syncthreads();
    for (int w = T / 2; w > 0; w >>= 1) {
        if (tid < w) red[tid] = fmax(red[tid], red[tid + w]);
        __syncthreads();
    }
    const double tn = red[0];
    if (bad || !isfinite(tn)) {
        if (tid == 0) {
            M.status = ST_ERR_NONFINITE;
            M.nblocks = 0;
        }
        return;
    }
    double scale = 1.0;
    if (tn > 0.0) {
        int ex;
        frexp(tn, &ex);
        scale = ldexp(1.0, -ex);
    }
    const double thresh = cfg.eps_x * tn;
    // rows [c0, c1) of this thread: scaled copy, split, block starts
    const int per = (n + T - 1) / T;
    const int c0 = min(n, tid * per), c1 = min(n, c0 + per);
    int starts = 0;
    for (int i = c0; i < c1; ++i) {
        wd[M.row0 + i] = ld_x<X>(M.d, i) * scale;
        if (i < n - 1) {
            double ei = ld_x<X>(M.e, i);
            we[M.row0 + i] = fabs(ei) <= thresh ? 0.0 : ei * scale;
        } else {
            we[M.row0 + i] = 0.0;
        }
        if (i == 0 || fabs(ld_x<X>(M.e, i - 1)) <= thresh) ++starts;
    }
    cnt[tid] = starts;
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int k = 0; k < T; ++k) {
            int v = cnt[k];
            cnt[k] = acc;
            acc += v;
        }
        M.nblocks = acc;
        M.scale = scale;
        M.tnorm = tn;
    }
    __syncthreads();
    int b = cnt[tid];
    for (int i = c0; i < c1; ++i) {
        if (i == 0 || fabs(ld_x<X>(M.e, i - 1)) <= thresh) {
            BlockDesc& B = blocks[M.row0 + b];
            B.matrix = blockIdx.x;
            B.row0 = M.row0 + i;
            B.mrow = i;
            ++b;
        }
    }
    __syncthreads();
    const int nb = M.nblocks;
    for (int k = tid; k < nb; k += T) {
        BlockDesc& B = blocks[M.row0 + k];
        int end = (k + 1 < nb) ? blocks[M.row0 + k + 1].mrow : n;
        B.n = end - B.mrow;
    }
}

// One CTA per block: the two candidate factorizations run on two warps, the
// perturbation and derived data on all threads.
// The leading principal minors of T - mu I for one root candidate, by one
// thread: P_i = (a_i - mu) P_{i-1} - b_{i-1}^2 P_{i-2} with P_{-1} = 1,
// P_{-2} = 0.  On entry D[i] = a_i - mu and L[i] = b_i^2; on exit D[i] = P_i,
// and the pair (P_{i-1}, P_{i-2}) carried to the next row is rescaled by a
// power of two (on the exponent fields) after every sixteenth row, whose
// rescaled P_i goes to L[i] -- so row i + 1 divides by L[i] after such a row
// and by D[i] after any other.  Two FP64 instructions per row on the chain.
constexpr int kMinorGroup = 16;
__device__ __forceinline__ void minor_chain(double* __restrict__ D, double* __restrict__ L, int n) {
    double pm1 = 1.0, pm2 = 0.0, e2 = 0.0;
    for (int i0 = 0; i0 < n; i0 += kMinorGroup) {
        double t[kMinorGroup], e[kMinorGroup];
#pragma unroll
        for (int k = 0; k < kMinorGroup; ++k) {
            const int i = min(i0 + k, n - 1);
            t[k] = D[i];
            e[k] = i < n - 1 ? L[i] : 0.0;
        }
        const int m = min(kMinorGroup, n - i0);
#pragma unroll
        for (int k = 0; k < kMinorGroup; ++k) {
            if (k < m) {
                const double P = fma(t[k], pm1, -(e2 * pm2));
                D[i0 + k] = P;
                pm2 = pm1;
                pm1 = P;
                e2 = e[k];
            }
        }
        const int q = dnotnormal(pm1) ? 0 : dscale_exp(pm1);
        pm1 = dscale_bits(pm1, q);
        pm2 = dscale_bits(pm2, q);
        if (m == kMinorGroup && i0 + m < n) L[i0 + m - 1] = pm1;
    }
}

// Both root candidates of k_root (Algorithm 1, line 2: L D L^T = T - mu I
// with mu just outside either end of the Gershgorin interval), in binary64,
// by the whole block.  One thread per side runs the minors' recurrence
// (minor_chain) on a_i - mu and b_i^2 formed beforehand by the block; then
// every thread forms d_i = P_i / P_{i-1} and l_i = b_i / d_i, the growth
// max |d_i| and the definiteness check (every pivot of the side's sign, none
// zero or non-finite).  A side that fails retries further out (delta x 16),
// as root_candidate does.  Rounding: d_i = P_i / P_{i-1} satisfies
// d_i = (a_i - mu) - b_{i-1}^2 / d_{i-1} with both terms perturbed by a few
// ulps, the mixed relative stability of the direct factorization; the random
// perturbation xi = 4 eps_x that follows (root_element) is larger.  Against
// one serial chain with a Newton reciprocal per row (about eight FP64
// instructions), the chain is two.  For double-double reps the binary64
// factors are then widened exactly, as in root_candidate.
template <class Y>
__device__ void root_candidates_block(const BlockDesc& B, const double* __restrict__ wd,
                                      const double* __restrict__ we, Y* reps, double gl, double gu, double* s_g,
                                      double* s_mu) {
    constexpr int T = kRootThreads;
    __shared__ double s_delta[2];
    __shared__ int s_need[2], s_bad[2];
    __shared__ unsigned long long s_gmax[2];
    const int n = B.n;
    const double* a = wd + B.row0;
    const double* b = we + B.row0;
    auto out = [&](int side) { return (double*)(reps + 4 * (size_t)B.row0 + (side ? 2 * (size_t)n : 0)); };
    auto mu_of = [&](int side) { return side ? gu + s_delta[side] : gl - s_delta[side]; };
    if (threadIdx.x < 2) {
        s_delta[threadIdx.x] = 4.0 * n * 1.1102230246251565e-16 * fmax(fabs(gl), fabs(gu)) + 4.0 * B.pivmin;
        s_need[threadIdx.x] = 1;
    }
    __syncthreads();
    for (int attempt = 0; attempt < 40; ++attempt) {
        const int need[2] = {s_need[0], s_need[1]};
        if (!need[0] && !need[1]) break;
        for (int side = 0; side < 2; ++side) {
            if (!need[side]) continue;
            const double mu = mu_of(side);
            double* D = out(side);
            for (int i = threadIdx.x; i < n; i += T) {
                D[i] = a[i] - mu;
                if (i < n - 1) D[n + i] = b[i] * b[i];
            }
        }
        if (threadIdx.x < 2) {
            s_bad[threadIdx.x] = 0;
            s_gmax[threadIdx.x] = 0ULL;
        }
        __syncthreads();
        if ((threadIdx.x == 0 && need[0]) || (threadIdx.x == 32 && need[1])) {
            double* D = out(threadIdx.x == 32);
            minor_chain(D, D + n, n);
        }
        __syncthreads();
        for (int side = 0; side < 2; ++side) {
            if (!need[side]) continue;
            double* D = out(side);
            double* L = D + n;
            const int want = side ? 1 : 0;  // sign bit of every pivot
            unsigned long long gmax = 0ULL;
            int bad = 0;
            // descending chunks: a chunk reads its own rows and the row below
            // it before any of them is overwritten
            for (int c0 = ((n - 1) / T) * T; c0 >= 0; c0 -= T) {
                const int i = c0 + threadIdx.x;
                double num = 0.0, den = 1.0;
                if (i < n) {
                    num = D[i];
                    if (i > 0) den = ((i - 1) % kMinorGroup == kMinorGroup - 1) ? L[i - 1] : D[i - 1];
                }
                __syncthreads();
                if (i < n) {
                    const double d = num / den;
                    const unsigned long long ab = dabsbits(d);
                    bad |= (dsign(d) != want) | (ab == 0ULL) | !dfinite(d);
                    gmax = ab > gmax ? ab : gmax;
                    D[i] = d;
                    L[i] = i < n - 1 ? b[i] / d : 0.0;
                }
                __syncthreads();
            }
            if (bad) atomicOr(&s_bad[side], 1);
            atomicMax(&s_gmax[side], gmax);
        }
        __syncthreads();
        if (threadIdx.x < 2 && need[threadIdx.x]) {
            const int side = threadIdx.x;
            if (!s_bad[side]) {
                s_g[side] = __longlong_as_double((long long)s_gmax[side]);
                s_mu[side] = mu_of(side);
                s_need[side] = 0;
            } else {
                s_delta[side] *= 16.0;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < 2 && s_need[threadIdx.x]) {
        s_g[threadIdx.x] = INFINITY;
        s_mu[threadIdx.x] = mu_of(threadIdx.x);
    }
    if constexpr (std::is_same<Y, dd>::value) {
        // widen both sides in place: double-double entry i covers binary64
        // words 2i, 2i+1 >= i, so descending chunks read before they write
        for (int side = 0; side < 2; ++side) {
            Y* rep = reps + 4 * (size_t)B.row0 + (side ? 2 * (size_t)n : 0);
            const double* src = (const double*)rep;
            for (int c0 = ((2 * n - 1) / T) * T; c0 >= 0; c0 -= T) {
                const int i = c0 + threadIdx.x;
                const double v = i < 2 * n ? src[i] : 0.0;
                __syncthreads();
                if (i < 2 * n) rep[i] = dd(v);
                __syncthreads();
            }
        }
    }
    __syncthreads();
}

template <class Y, class Lo>
__global__ void k_root(const int* blist, BlockDesc* blocks, const MatrixDesc* mats, const double* wd,
                       const double* we, Y* reps, Lo* reps_lo, SolveCfg cfg) {
    constexpr int T = kRootThreads;
    __shared__ double s_gl, s_gu, s_g[2], s_mu[2];
    __shared__ double r_gl[T], r_gu[T], r_e2[T];
    BlockDesc& B = blocks[blist[blockIdx.x]];
    const MatrixDesc& M = mats[B.matrix];
    const int n = B.n;
    {
        // Gershgorin bounds: strided partials, then a tree reduction
        double gl = INFINITY, gu = -INFINITY, e2 = 0.0;
        root_bounds_part(B, wd, we, threadIdx.x, T, &gl, &gu, &e2);
        r_gl[threadIdx.x] = gl;
        r_gu[threadIdx.x] = gu;
        r_e2[threadIdx.x] = e2;
        __syncthreads();
        for (int h = T / 2; h > 0; h >>= 1) {
            if (threadIdx.x < h) {
                r_gl[threadIdx.x] = fmin(r_gl[threadIdx.x], r_gl[threadIdx.x + h]);
                r_gu[threadIdx.x] = fmax(r_gu[threadIdx.x], r_gu[threadIdx.x + h]);
                r_e2[threadIdx.x] = fmax(r_e2[threadIdx.x], r_e2[threadIdx.x + h]);
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            root_bounds_finish<Y>(B, r_gl[0], r_gu[0], r_e2[0]);
            s_gl = r_gl[0];
            s_gu = r_gu[0];
        }
        __syncthreads();
    }
    if (n == 1) {
        if (threadIdx.x == 0) {
            root_trivial<Y, Lo>(B, wd, reps, reps_lo);
            root_range<Y>(B, M, wd, reps);
        }
        return;
    }
    if constexpr (std::is_same<Y, double>::value || std::is_same<Y, dd>::value) {
        root_candidates_block<Y>(B, wd, we, reps, s_gl, s_gu, s_g, s_mu);
    } else {
        if (threadIdx.x == 0 || threadIdx.x == 32) {
            int side = threadIdx.x == 32;
            s_g[side] = root_candidate<Y>(B, wd, we, reps, s_gl, s_gu, side, &s_mu[side]);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) root_choose(B, M, s_gl, s_gu, s_g[0], s_mu[0], s_g[1], s_mu[1], cfg);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) root_move<Y>(B, reps, i);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) root_element<Y, Lo>(B, M, reps, reps_lo, i, cfg, we);
    __syncthreads();
    if (threadIdx.x == 0) root_range<Y>(B, M, wd, reps);
}

// Exclusive scan of the item counts over the block list (one CTA), plus the
// per-matrix totals: item range, number of returned eigenpairs.
static __global__ void k_scan_items(const int* blist, int nb, BlockDesc* blocks, MatrixDesc* mats, int nmat,
                                    int* total_out) {
    __shared__ int part[1024];
    const int T = blockDim.x;
    int per = (nb + T - 1) / T;
    int b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
    int s = 0;
    for (int b = b0; b < b1; ++b) s += blocks[blist[b]].nitems;
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int i = 0; i < T; ++i) {
            int v = part[i];
            part[i] = acc;
            acc += v;
        }
        *total_out = acc;
    }
    __syncthreads();
    int off = part[threadIdx.x];
    for (int b = b0; b < b1; ++b) {
        BlockDesc& B = blocks[blist[b]];
        B.item0 = off;
        off += B.nitems;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < nmat; p += T) {
        MatrixDesc& M = mats[p];
        int item0 = -1, nit = 0, kout = 0;
        for (int b = 0; b < M.nblocks; ++b) {
            const BlockDesc& B = blocks[M.row0 + b];
            if (item0 < 0 && B.nitems > 0) item0 = B.item0;
            nit += B.nitems;
            if (B.w_hi >= B.w_lo) kout += B.w_hi - B.w_lo + 1;
        }
        if (M.range == RANGE_INDEX && M.nblocks > 0) kout = M.iu - M.il + 1;
        M.item0 = item0 < 0 ? 0 : item0;
        M.nitems = nit;
        M.kout = M.nblocks > 0 ? kout : 0;
    }
}

// One thread per item; the block is found by binary search over the item
// offsets (ascending in block-list order).
template <class Y, class Lo>
__global__ void k_init_items(const int* blist, int nb, const BlockDesc* blocks, Item* items, int K, const Y* reps,
                             const Lo* reps_lo) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= K) return;
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (blocks[blist[mid]].item0 <= t) lo = mid;
        else hi = mid - 1;
    }
    // skip blocks without items that share the same offset
    while (lo + 1 < nb && blocks[blist[lo]].nitems == 0) ++lo;
    const BlockDesc& B = blocks[blist[lo]];
    init_item<Y, Lo>(B, blist[lo], items[t], t - B.item0, reps, reps_lo);
}

template <class Y>
__global__ void k_bisect(Item* items, const int* list, int count, const int* count_dev, const BlockDesc* blocks,
                         double rtol, int verify, unsigned long long* step_counter) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (count_dev) count = *count_dev;
    if (t >= count) return;
    int it = list ? list[t] : t;
    Item& I = items[it];
    unsigned long long steps = 0;
    bisect_item<Y>(I, blocks[I.block].pivmin, rtol, verify, 200, &steps);
    if (steps) atomicAdd(step_counter, steps);
}

template <class Lo>
__global__ void k_bisect_lo(Item* items, const int* list, int count, const BlockDesc* blocks, double wrel,
                            DevCounters* C) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    Item& I = items[list ? list[t] : t];
    unsigned long long s = bisect_lo_item<Lo>(I, blocks[I.block].pivmin, wrel, 200);
    if (s) atomicAdd(&C->qd_steps_low, s);
}

// Multisection sweeps (kMS, ms_point) with the lanes of one item adjacent in
// a warp, sharing their counts by shuffles.

// shuffle mask of the M-lane group of this thread
template <int M = kMS>
__device__ __forceinline__ unsigned ms_mask() {
    return ((1u << M) - 1u) << ((threadIdx.x & 31) & ~(M - 1));
}

// point q of an M-point multisection sweep of [lo, hi]
template <int M>
__device__ __forceinline__ double ms_point_m(double lo, double hi, int q) {
    return lo + (hi - lo) / (M + 1) * (q + 1);
}

// Given the counts c_k at the points x_k (k < kMS) of a sweep, in increasing
// order: the first point whose count reaches j is the new upper end and the
// point before it the new lower end -- well defined even where rounding makes
// a count non-monotone.  Points that rounded onto or outside the bracket are
// skipped.  Returns false when no point was inside.
template <int M = kMS>
__device__ __forceinline__ bool ms_update(unsigned mask, int c, double x, bool inside, int j, double& lo, double& hi) {
    double nlo = lo, nhi = hi;
    bool any_inside = false, found = false;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const int ck = __shfl_sync(mask, c, k, M);
        const double xk = __shfl_sync(mask, x, k, M);
        const bool ik = __shfl_sync(mask, (int)inside, k, M) != 0;
        any_inside |= ik;
        if (!ik || found) continue;
        if (ck >= j) {
            nhi = xk;
            found = true;
        } else {
            nlo = xk;
        }
    }
    if (!any_inside) return false;
    lo = nlo;
    hi = nhi;
    return true;
}

// Low-precision pre-bisection of the listed items (Sec. 3.2: eigenvalues are
// approximated in a precision below the working one) down to a relative
// width wrel, by multisection with M lanes per item.
template <class Lo, int M>
__global__ void k_bisect_lo_ms(Item* items, const int* list, int count, const BlockDesc* blocks, double wrel,
                               DevCounters* C) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int g = t / M, q = t % M;
    if (g >= count) return;  // whole groups leave together (M divides 32)
    const unsigned mask = ms_mask<M>();
    Item& I = items[list ? list[g] : g];
    const int n = I.n;
    if (n == 1) return;
    const Lo* D = (const Lo*)I.rep_lo;
    const Lo* LLD = D + n;
    Lo pm = (Lo)fmax(blocks[I.block].pivmin, (double)Prec<Lo>::tiny * 4.0);
    double lo = I.lo, hi = I.hi;
    unsigned long long steps = 0;
    for (int it = 0; it < 64; ++it) {
        if (!(hi - lo > wrel * fmax(fabs(lo), fabs(hi)))) break;
        const Lo x = (Lo)ms_point_m<M>(lo, hi, q);
        const bool inside = (double)x > lo && (double)x < hi;
        const int c = inside ? count_lo<Lo>(D, LLD, n, x, pm) : 0;
        if (inside) steps += (unsigned long long)n;
        if (!ms_update<M>(mask, c, (double)x, inside, I.j, lo, hi)) break;  // no representable interior point left
    }
    if (q == 0) {
        I.lo = lo;
        I.hi = hi;
    }
    if (steps) atomicAdd(&C->qd_steps_low, steps);
}

// Working-precision refinement of the listed items by multisection (the
// same sweeps as k_bisect_lo_ms, with the count of the working precision):
// down to hi - lo <= max(rtol max(|lo|, |hi|), 2 pivmin), as bisect_bracket.
// The refinement starts from verified brackets a few bits wide.  The list
// length is read on the device.
template <class Y>
__global__ void k_bisect_ms(Item* items, const int* list, const int* count_dev, int bound, const BlockDesc* blocks,
                            double rtol, unsigned long long* step_counter) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int g = t / kMS, q = t % kMS;
    if (g >= bound || g >= *count_dev) return;  // whole groups leave together (kMS divides 32)
    const unsigned mask = ms_mask();
    Item& I = items[list[g]];
    const int n = I.n;
    if (n == 1) {
        if (q == 0) {
            I.lo = 0.0;
            I.hi = 0.0;
        }
        return;
    }
    const Y* D = (const Y*)I.rep;
    const Y* LLD = D + 3 * n;
    const double pivmin = blocks[I.block].pivmin;
    const Y pm = from_d<Y>(pivmin);
    double lo = I.lo, hi = I.hi;
    unsigned long long steps = 0;
    for (int it = 0; it < 64; ++it) {
        const double tol = fmax(rtol * fmax(fabs(lo), fabs(hi)), 2.0 * pivmin);
        if (!(tol < hi - lo)) break;
        const double x = ms_point(lo, hi, q);
        const bool inside = x > lo && x < hi;
        const int c = inside ? count_at<Y, true>(D, LLD, n, from_d<Y>(x), pm) : 0;
        if (inside) steps += (unsigned long long)n;
        if (!ms_update(mask, c, x, inside, I.j, lo, hi)) break;
    }
    if (q == 0) {
        I.lo = lo;
        I.hi = hi;
    }
    if (steps) atomicAdd(step_counter, steps);
}

// Two threads per item, one per end of the bracket: one working-precision
// count each.  An end that fails marks its item (bit `side` of vflags); the
// first of the two to mark it appends the item to fix_list, so that the few
// items whose ends must move run in a separate, densely packed launch
// instead of holding a whole warp here.
template <class Y>
__global__ void k_verify(Item* items, const int* list, int count, const BlockDesc* blocks, DevCounters* C,
                         unsigned long long* step_counter, int* vflags, int* fix_list) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * count) return;
    int it = list ? list[t >> 1] : (t >> 1);
    const Item& I = items[it];
    if (I.n == 1) return;
    const int side = t & 1;
    int c = endpoint_count<Y>(I, blocks[I.block], side);
    atomicAdd(step_counter, (unsigned long long)I.n);
    if (!endpoint_holds(I, side, c) && atomicOr(&vflags[it], 1 << side) == 0) fix_list[atomicAdd(&C->nvfix, 1)] = it;
}

// kFixLanes lanes per listed item move its failing ends.  For a failing
// lower end x (count(x) >= j) the lanes test, in one sweep, the points
// x - w 4^k for k = 0..kFixLanes-1; the point nearest to x whose count is < j
// is the new lower end, and the point tested just before it -- whose count
// is still >= j, so it bounds lambda_j from above -- the new upper end when
// that end did not fail too.  Symmetrically for a failing upper end.  w is
// the first doubling step of the sequential check (endpoint_step), so the
// sweep covers fourteen doublings with the latency of one count (the first
// point, one bracket width out, is where most ends that failed end up).  Beyond
// that the end falls back to the sequential widening, which ends at the
// bound of the whole spectrum.
constexpr int kFixLanes = 8;
// lanes per item of the low-precision pre-bisection: kMSRoot at the root
// level; kMSChild for cluster members in their child rep, which start from
// brackets many orders of magnitude wider than their eigenvalues (the
// parent's brackets, shifted) -- sixteen points per sweep take fewer sweeps,
// and leave brackets from which fewer eigenpairs need a third RQI step
// (measured on the n = 4001 step: 15.0 ms against 15.7 ms with four; eight
// or sixteen at the root level made the RQI slower).  Only while the list is
// short enough to leave SM sub-partitions idle, and only for a binary32
// count: a batch of thousands of matrices (6.0M against 6.4M eigenpairs/s)
// and the binary64 pre-bisection of the double-double solver were slower
// with sixteen.
constexpr int kMSRoot = kMS;
constexpr int kMSChild = 16;
constexpr int kMSChildMaxItems = 32768;
constexpr int kFixSweeps = 1;
template <class Y>
__global__ void k_verify_fix(Item* items, const int* fix_list, int bound, const BlockDesc* blocks, DevCounters* C,
                             unsigned long long* step_counter, int* vflags) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int g = t / kFixLanes, q = t % kFixLanes;
    if (g >= bound || g >= C->nvfix) return;  // whole groups leave together (kFixLanes divides 32)
    unsigned mask = ((1u << kFixLanes) - 1u) << ((threadIdx.x & 31) & ~(kFixLanes - 1));
    const int it = fix_list[g];
    Item& I = items[it];
    const BlockDesc& B = blocks[I.block];
    const int m = vflags[it];
    const int n = I.n;
    const Y* rep = (const Y*)I.rep;
    const Y pm = from_d<Y>(B.pivmin);
    const double w0[2] = {endpoint_step(I, B, 0), endpoint_step(I, B, 1)};
    double x[2] = {I.lo, I.hi};
    unsigned long long steps = 0;
    int fails = 0;
    for (int side = 0; side < 2; ++side) {
        if (!(m & (1 << side))) continue;
        const double x0 = side ? I.hi : I.lo;
        double last_fail = x0;  // nearest tested point known to fail
        bool found = false;
        double p = x0;
        for (int sw = 0; sw < kFixSweeps && !found; ++sw) {
            double f = ldexp(1.0, 2 * (sw * kFixLanes + q));  // 4^(k-1)
            double xq = side ? x0 + w0[side] * f : x0 - w0[side] * f;
            int c = count_at<Y, true>(rep, rep + 3 * n, n, from_d<Y>(xq), pm);
            steps += (unsigned long long)n;
            bool ok = endpoint_holds(I, side, c);
#pragma unroll
            for (int k = 0; k < kFixLanes; ++k) {
                bool okk = __shfl_sync(mask, (int)ok, k, kFixLanes) != 0;
                double xk = __shfl_sync(mask, xq, k, kFixLanes);
                if (found) continue;
                if (okk) {
                    found = true;
                    p = xk;
                } else {
                    last_fail = xk;
                }
            }
        }
        fails += found ? 1 : 0;
        if (!found) {
            // sequential widening from the last failing point
            Item J = I;
            if (side) J.hi = last_fail;
            else J.lo = last_fail;
            p = widen_endpoint<Y>(J, B, side, w0[side] * ldexp(1.0, 2 * kFixSweeps * kFixLanes), &steps, &fails);
        }
        x[side] = p;
        // the last failing point bounds lambda_j on the other side
        if (!(m & (1 << (1 - side)))) x[1 - side] = side ? fmax(x[0], last_fail) : fmin(x[1], last_fail);
    }
    if (q == 0) {
        I.lo = x[0];
        I.hi = x[1];
        vflags[it] = 0;
        atomicAdd(&C->verify_fail, fails);
    }
    if (steps) atomicAdd(step_counter, steps);
}

static __global__ void k_certify(const Item* items, int K, const int* list, int count, double gaptol,
                                 int* refine_list, DevCounters* C) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    int it = list ? list[t] : t;
    if (!certified(it, items, K, gaptol)) {
        int slot = atomicAdd(&C->nrefine, 1);
        refine_list[slot] = it;
    }
}

static __global__ void k_assign_cols(Item* items, int count, const MatrixDesc* mats, const BlockDesc* blocks) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    assign_col(t, items, mats, blocks);
}

// One thread per item of the list (all items at the root level, the members
// of the previous level's clusters below it).
static __global__ void k_classify(Item* items, const int* list, int count, int K, double gaptol, int* single_list,
                                  Cluster* clusters, int* member_list, DevCounters* C) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    classify_item(list ? list[t] : t, items, K, gaptol, single_list, clusters, member_list, C);
}

template <class Y, class Lo>
__global__ void k_shift(const Cluster* clusters, int nc, Item* items, const BlockDesc* blocks, Y* pool, Lo* pool_lo,
                        SolveCfg cfg, DevCounters* C) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nc) return;
    shift_cluster<Y, Lo>(clusters[t], items, blocks, pool, pool_lo, cfg, C);
}

// Persistent RQI over a list of eigenpairs: one-warp CTAs, each warp takes
// the next 32 entries of the list from a global counter (`queue`) until the
// list is exhausted, so warps that finish early keep taking work and the
// scratch belongs to the warp (2 nmax working-precision words per lane), not
// to the eigenpair -- a batch of any size runs in one launch.  One thread
// per eigenpair: at most pass_iters RQI steps; unfinished eigenpairs go to
// park_list.  Finished vectors are written by the whole warp: a 32 x 32
// tile (32 rows of the 32 lanes' vectors) goes through shared memory so that
// each column segment is one contiguous 128-byte (binary32) / 256-byte
// (binary64) store, instead of 32 scattered words per instruction.
template <class X, class Y>
__global__ void k_rqi(Item* items, const int* list, int count, const int* dev_total, int* queue, MatrixDesc* mats,
                      const BlockDesc* blocks, SolveCfg cfg, Y* scratch, int nmax, DevCounters* C, int pass_iters,
                      int final_pass, int* park_list, int* park_count) {
    constexpr bool kCoop = !std::is_same<Y, dd>::value;
    __shared__ X tile[32][33];
    __shared__ X* col_of[32];
    __shared__ int rows_of[32];
    const int lane = threadIdx.x & 31;
    // this warp's scratch slot (one-warp CTAs), reused for every chunk it takes
    Y* base = scratch + ((size_t)blockIdx.x * 32 + lane) * (size_t)(2 * nmax);
    Scratch<Y> Wk;
    Wk.a = base;
    Wk.b = base + nmax;
    Wk.stride = 1;
    // a later pass is launched for an upper bound and reads the true length
    // of its list on the device
    const int total = dev_total ? min(count, *dev_total) : count;
    for (;;) {
        int b0 = 0;
        if (lane == 0) b0 = atomicAdd(queue, 32);
        b0 = __shfl_sync(0xffffffffu, b0, 0);
        if (b0 >= total) break;
        const int t = b0 + lane;
        const bool active = t < total;
        const int it = active ? list[t] : 0;
        double scale = 0.0;
        bool stored = false;
        if (active) {
            Item& I = items[it];
            stored = rqi_item<X, Y>(I, mats, blocks, cfg, Wk, C, pass_iters, final_pass != 0,
                                    kCoop ? &scale : nullptr);
            if (!stored) {
                int slot = atomicAdd(park_count, 1);
                park_list[slot] = it;
            }
        }
        if constexpr (kCoop) {
            // warp-cooperative store of the finished vectors
            int nrow = 0;
            X* col = nullptr;
            if (stored) {
                const Item& I = items[it];
                const MatrixDesc& M = mats[I.matrix];
                nrow = I.n;
                col = (X*)M.Z + (size_t)I.outcol * (size_t)M.ldz + blocks[I.block].mrow;
            }
            int nmaxw = nrow;
            for (int o = 16; o > 0; o >>= 1) nmaxw = max(nmaxw, __shfl_xor_sync(0xffffffffu, nmaxw, o));
            // every lane's column and length, read back by the whole warp
            col_of[lane] = col;
            rows_of[lane] = nrow;
            __syncwarp();
            for (int r0 = 0; r0 < nmaxw; r0 += 32) {
                // lane l: rows r0..r0+31 of its own vector into tile row l
                // (all 32 loads issued before the first use)
                double v[32];
#pragma unroll
                for (int q = 0; q < 32; ++q) v[q] = (r0 + q < nrow) ? to_d(Wk.a[r0 + q]) : 0.0;
#pragma unroll
                for (int q = 0; q < 32; ++q) tile[lane][q] = (X)(v[q] * scale);
                __syncwarp();
                // column c of the tile: lanes write 32 consecutive rows
#pragma unroll 8
                for (int c = 0; c < 32; ++c) {
                    X* cc = col_of[c];
                    const int r = r0 + lane;
                    if (cc && r < rows_of[c]) cc[r] = tile[c][lane];
                }
                __syncwarp();
            }
            __syncwarp();
        }
    }
}

// Ordering of W for matrices that split.  Eigenvalues of different blocks
// were given their columns by bracket midpoints; the final values can order
// differently where they agree to rounding (identical blocks give ties).
// k_rank: the position of each eigenvalue in ascending order, stable (equal
// values keep their column order, NaN sorts last), by counting, one thread
// per eigenvalue with the values staged through shared memory in tiles;
// flag[y] is set when the matrix is not in order yet.  Then k_gather moves
// column i to column rank(i) of a temporary and k_copy_back copies it back.
constexpr int kRankTile = 256;
template <class X>
__global__ void k_rank(const MatrixDesc* mats, const int* list, const long long* roff, int* rank, int* flag) {
    __shared__ X tile[kRankTile];
    const MatrixDesc& M = mats[list[blockIdx.y]];
    const int k = M.kout;
    const int i = blockIdx.x * kRankTile + threadIdx.x;
    if (blockIdx.x * kRankTile >= k) return;  // whole CTA leaves together
    const X* W = (const X*)M.W;
    const X wi = i < k ? W[i] : X(0);
    const bool ni = !(wi == wi);
    int r = 0;
    for (int j0 = 0; j0 < k; j0 += kRankTile) {
        __syncthreads();
        if (j0 + threadIdx.x < k) tile[threadIdx.x] = W[j0 + threadIdx.x];
        __syncthreads();
        const int jn = min(kRankTile, k - j0);
        if (i < k) {
            for (int q = 0; q < jn; ++q) {
                const X wj = tile[q];
                const int j = j0 + q;
                const bool nj = !(wj == wj);
                r += ni ? (!nj || j < i) : (!nj && (wj < wi || (wj == wi && j < i)));
            }
        }
    }
    if (i < k) {
        rank[roff[blockIdx.y] + i] = r;
        if (r != i) flag[blockIdx.y] = 1;
    }
}

// CTA (x = column, y = listed matrix): column x of Z (and W[x]) to column
// rank(x) of the temporary T (leading dimension n) and Wt.
template <class X>
__global__ void k_gather(const MatrixDesc* mats, const int* list, const long long* roff, const int* rank,
                         const long long* toff, X* T, X* Wt) {
    const MatrixDesc& M = mats[list[blockIdx.y]];
    const int c = blockIdx.x;
    if (c >= M.kout) return;
    const int dst = rank[roff[blockIdx.y] + c];
    const X* src = (const X*)M.Z + (size_t)c * M.ldz;
    X* out = T + toff[blockIdx.y] + (size_t)dst * M.n;
    for (int r = threadIdx.x; r < M.n; r += blockDim.x) out[r] = src[r];
    if (threadIdx.x == 0) Wt[roff[blockIdx.y] + dst] = ((const X*)M.W)[c];
}

template <class X>
__global__ void k_copy_back(const MatrixDesc* mats, const int* list, const long long* roff, const long long* toff,
                            const X* T, const X* Wt) {
    const MatrixDesc& M = mats[list[blockIdx.y]];
    const int c = blockIdx.x;
    if (c >= M.kout) return;
    X* dst = (X*)M.Z + (size_t)c * M.ldz;
    const X* src = T + toff[blockIdx.y] + (size_t)c * M.n;
    for (int r = threadIdx.x; r < M.n; r += blockDim.x) dst[r] = src[r];
    if (threadIdx.x == 0) ((X*)M.W)[c] = Wt[roff[blockIdx.y] + c];
}

// ------------------------------------------------------------------ host driver

// Stream-ordered allocations from the library's pool, released together at
// the end of a solve.
struct Arena {
    cudaStream_t st;
    std::vector<void*> ptrs;
    bool failed = false;
    explicit Arena(cudaStream_t s) : st(s) {}
    template <class T> T* alloc(size_t count) {
        void* p = dev_alloc(std::max<size_t>(count, 1) * sizeof(T), st);
        if (!p) {
            failed = true;
            return nullptr;
        }
        ptrs.push_back(p);
        return (T*)p;
    }
    ~Arena() {
        for (void* p : ptrs) dev_free(p, st);
    }
};

// Pinned host staging for one solve: every block handed out stays valid
// until the solve returns, so an upload never has to wait for its copy.
struct HostArena {
    std::vector<std::pair<void*, size_t>> blocks;
    bool failed = false;
    template <class T> T* get(size_t count) {
        size_t got = 0;
        void* p = host_alloc(std::max<size_t>(count, 1) * sizeof(T), &got);
        if (!p) {
            failed = true;
            return nullptr;
        }
        blocks.emplace_back(p, got);
        return (T*)p;
    }
    ~HostArena() {
        for (auto& b : blocks) host_free(b.first, b.second);
    }
};

// Copies between host data and the device through pinned staging.
template <class T>
int to_device(HostArena& ha, T* dst, const T* src, size_t count, cudaStream_t st) {
    T* h = ha.get<T>(count);
    if (!h) return MRRR_ERR_NOMEM;
    memcpy(h, src, sizeof(T) * count);
    return cudaMemcpyAsync(dst, h, sizeof(T) * count, cudaMemcpyHostToDevice, st) == cudaSuccess ? 0 : MRRR_ERR_CUDA;
}

template <class T>
int from_device(HostArena& ha, T* dst, const T* src, size_t count, cudaStream_t st) {
    T* h = ha.get<T>(count);
    if (!h) return MRRR_ERR_NOMEM;
    if (cudaMemcpyAsync(h, src, sizeof(T) * count, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return MRRR_ERR_CUDA;
    memcpy(dst, h, sizeof(T) * count);
    return 0;
}

#define MRRR_CK(call)                                  \
    do {                                               \
        cudaError_t err__ = (call);                    \
        if (err__ != cudaSuccess) return MRRR_ERR_CUDA; \
    } while (0)

#define MRRR_ALLOC(var, T, count)                       \
    T* var = arena.alloc<T>(count);                     \
    if (!var) return MRRR_ERR_NOMEM

// Optional per-phase device timing with CUDA events on the solve's stream.
struct Timeline {
    bool on;
    cudaStream_t st;
    struct Rec {
        int phase, launches;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    cudaEvent_t cur_a = nullptr;
    int cur = -1;
    Timeline(bool enabled, cudaStream_t s) : on(enabled), st(s) {}
    void begin(int phase, cudaStream_t s = nullptr) {
        if (!on) return;
        cudaEventCreate(&cur_a);
        cudaEventRecord(cur_a, s ? s : st);
        cur = phase;
    }
    void end(int launches = 1, cudaStream_t s = nullptr) {
        if (!on) return;
        cudaEvent_t b;
        cudaEventCreate(&b);
        cudaEventRecord(b, s ? s : st);
        recs.push_back({cur, launches, cur_a, b});
    }
    void collect(mrrr_stats* s) {
        for (Rec& r : recs) {
            float ms = 0.f;
            if (s && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
                s->phase_ms[r.phase] += ms;
                s->phase_launches[r.phase] += r.launches;
            }
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        recs.clear();
        if (s) s->timed = on ? 1 : 0;
    }
    ~Timeline() { collect(nullptr); }
};

// A second stream for work that may overlap the main stream; joined back
// into the main stream before the owner's allocations are released.
struct SideStream {
    cudaStream_t main;
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    explicit SideStream(cudaStream_t m) : main(m) {}
    bool start() {
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return false;
        if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess) return false;
        if (cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess) return false;
        if (cudaEventRecord(fork, main) != cudaSuccess) return false;
        return cudaStreamWaitEvent(s, fork, 0) == cudaSuccess;
    }
    void rejoin() {
        if (!s) return;
        cudaEventRecord(join, s);
        cudaStreamWaitEvent(main, join, 0);
    }
    ~SideStream() {
        if (s) {
            rejoin();
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
    }
};

template <class Y> struct ScratchBudget {
    static size_t bytes() { return (size_t)4 << 30; }  // 4 GiB of RQI scratch per wave
};

// Solve a batch of independent tridiagonals (a single solve is a batch of
// one).  mats[p] carries the input/output device pointers, n, ldz and range;
// the remaining fields are filled in.  Returns 0 or a negative status; the
// per-matrix status and count are left in mats[p].status / mats[p].kout.
// An autotuner trial: the RQI passes of one run, bracketed by two events.
struct TuneRun {
    unsigned key;
    int trial;
    cudaEvent_t a, b;
};

template <class X, class Y>
int solve_batch(int P, MatrixDesc* mats, const SolveCfg& cfg, int max_depth, cudaStream_t st,
                mrrr_stats* stats, RootSep* root_sep = nullptr) {
    typedef typename LowOf<Y>::T Lo;
    const bool use_low = LowOf<Y>::use && !(cfg.flags & MRRR_FLAG_NO_LOWPREC_BISECT);
    // relative width of the low-precision pre-bisection
    // relative width at which the low-precision pre-bisection stops: about
    // 8 units of binary32 at the root level (the brackets that pass the
    // working-precision check go to the RQI as they are, and a narrower one
    // needs fewer RQI steps), about 32 units below it
    const double wrel_lo = std::is_same<Lo, float>::value ? 0x1p-19 : cfg.rtol_class;
    const double wrel_root = std::is_same<Lo, float>::value ? 0x1p-21 : cfg.rtol_class;
    long long N = 0;
    int nmax = 1;
    for (int p = 0; p < P; ++p) {
        mats[p].row0 = (int)N;
        mats[p].status = ST_OK;
        mats[p].nblocks = 0;
        mats[p].kout = 0;
        N += mats[p].n;
        nmax = std::max(nmax, mats[p].n);
    }
    if (N > (1LL << 30) / 4) return MRRR_ERR_ARG;
    Arena arena(st);
    SideStream side(st);  // destroyed (joined) before the arena frees
    Timeline tl(stats && (cfg.flags & MRRR_FLAG_TIMING), st);
    MRRR_ALLOC(d_mats, MatrixDesc, P);
    MRRR_ALLOC(d_blocks, BlockDesc, N);
    MRRR_ALLOC(wd, double, N);
    MRRR_ALLOC(we, double, N);
    MRRR_ALLOC(reps, Y, 4 * N);
    MRRR_ALLOC(reps_lo, Lo, 2 * N);
    MRRR_ALLOC(d_C, DevCounters, 1);
    MRRR_ALLOC(d_total, int, 1);
    MRRR_CK(cudaMemsetAsync(d_C, 0, sizeof(DevCounters), st));
    HostArena ha;
    if (int rc0 = to_device(ha, d_mats, mats, (size_t)P, st)) return rc0;

    // a1: scale + split
    tl.begin(MRRR_PHASE_PREP);
    k_prep<X><<<P, 256, 0, st>>>(d_mats, d_blocks, wd, we, cfg);
    tl.end();
    MRRR_CK(cudaGetLastError());
    if (int rc0 = from_device(ha, mats, d_mats, (size_t)P, st)) return rc0;
    std::vector<int> blist;
    for (int p = 0; p < P; ++p)
        for (int b = 0; b < mats[p].nblocks; ++b) blist.push_back(mats[p].row0 + b);
    const int NB = (int)blist.size();
    DevCounters C{};
    int rqi_wps = 0, rqi_wps_list = 0;
    std::vector<TuneRun> tune_runs;  // timed autotuner trials, reported after the final synchronisation
    if (NB > 0) {
        MRRR_ALLOC(d_blist, int, NB);
        if (int rc0 = to_device(ha, d_blist, blist.data(), (size_t)NB, st)) return rc0;
        // a2: root representations
        tl.begin(MRRR_PHASE_ROOT);
        k_root<Y, Lo><<<NB, kRootThreads, 0, st>>>(d_blist, d_blocks, d_mats, wd, we, reps, reps_lo, cfg);
        k_scan_items<<<1, 1024, 0, st>>>(d_blist, NB, d_blocks, d_mats, P, d_total);
        tl.end(2);
        MRRR_CK(cudaGetLastError());
        int K = 0;
        if (int rc0 = from_device(ha, &K, d_total, 1, st)) return rc0;
        if (int rc0 = from_device(ha, mats, d_mats, (size_t)P, st)) return rc0;
        if (K > 0) {
            MRRR_ALLOC(items, Item, K);
            MRRR_ALLOC(single_list, int, K);
            MRRR_ALLOC(member_a, int, K);
            MRRR_ALLOC(member_b, int, K);
            MRRR_ALLOC(refine_list, int, K);
            MRRR_ALLOC(vfix_list, int, K);
            MRRR_ALLOC(vflags, int, K);
            MRRR_CK(cudaMemsetAsync(vflags, 0, sizeof(int) * (size_t)K, st));  // each fix launch clears what it used
            MRRR_ALLOC(clus_a, Cluster, K / 2 + 1);
            MRRR_ALLOC(clus_b, Cluster, K / 2 + 1);
            tl.begin(MRRR_PHASE_ROOT);
            k_init_items<Y, Lo><<<grid_for(K), kThreads, 0, st>>>(d_blist, NB, d_blocks, items, K, reps, reps_lo);
            tl.end();
            // eigenvector columns of a split matrix are zero outside their block
            tl.begin(MRRR_PHASE_FINISH);
            int nz = 0;
            for (int p = 0; p < P && !root_sep; ++p) {
                if (mats[p].nblocks > 1 && mats[p].kout > 0) {
                    MRRR_CK(cudaMemset2DAsync(mats[p].Z, sizeof(X) * (size_t)mats[p].ldz, 0,
                                              sizeof(X) * (size_t)mats[p].n, mats[p].kout, st));
                    ++nz;
                }
            }
            tl.end(nz);
            int num_sms = 0, dev = 0;
            if (cudaGetDevice(&dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || num_sms < 1)
                num_sms = 152;
            // a3: initial eigenvalues (Algorithm 1, line 3): low-precision
            // pre-bisection, verification of both bracket ends and refinement of
            // the items not yet certified, in the working precision
            auto approximate = [&](const int* list, int count, bool verify_ws, unsigned long long* ctr,
                                   int phase) -> int {
                tl.begin(phase);
                int launches = 0;
                if (use_low) {
                    if (phase == MRRR_PHASE_BISECT)
                        k_bisect_lo_ms<Lo, kMSRoot><<<grid_for((long long)count * kMSRoot, kLatThreads), kLatThreads,
                                                       0, st>>>(items, list, count, d_blocks, wrel_root, d_C);
                    else if (std::is_same<Lo, float>::value && count <= kMSChildMaxItems)
                        k_bisect_lo_ms<Lo, kMSChild><<<grid_for((long long)count * kMSChild, kLatThreads), kLatThreads, 0,
                                                        st>>>(items, list, count, d_blocks, wrel_lo, d_C);
                    else
                        k_bisect_lo_ms<Lo, kMS><<<grid_for((long long)count * kMS, kLatThreads), kLatThreads, 0, st>>>(
                            items, list, count, d_blocks, wrel_lo, d_C);
                    MRRR_CK(cudaMemsetAsync(&d_C->nvfix, 0, sizeof(int), st));
                    k_verify<Y><<<grid_for(2LL * count, kLatThreads), kLatThreads, 0, st>>>(
                        items, list, count, d_blocks, d_C, ctr, vflags, vfix_list);
                    k_verify_fix<Y><<<grid_for((long long)count * kFixLanes, kLatThreads), kLatThreads, 0, st>>>(
                        items, vfix_list, count, d_blocks, d_C, ctr, vflags);
                    MRRR_CK(cudaMemsetAsync(&d_C->nrefine, 0, sizeof(int), st));
                    k_certify<<<grid_for(count), kThreads, 0, st>>>(items, K, list, count, cfg.gaptol, refine_list,
                                                                    d_C);
                    k_bisect_ms<Y><<<grid_for((long long)count * kMS, kLatThreads), kLatThreads, 0, st>>>(
                        items, refine_list, &d_C->nrefine, count, d_blocks, cfg.rtol_class, ctr);
                    launches = 5;
                } else {
                    k_bisect<Y><<<grid_for(count, kLatThreads), kLatThreads, 0, st>>>(items, list, count, nullptr, d_blocks,
                                                                       cfg.rtol_class, verify_ws ? 1 : 0, ctr);
                    launches = 1;
                }
                tl.end(launches);
                return cudaGetLastError() == cudaSuccess ? 0 : MRRR_ERR_CUDA;
            };
            if (approximate(nullptr, K, false, &d_C->qd_bisect, MRRR_PHASE_BISECT)) return MRRR_ERR_CUDA;
            tl.begin(MRRR_PHASE_CLASSIFY);
            k_assign_cols<<<grid_for(K), kThreads, 0, st>>>(items, K, d_mats, d_blocks);
            tl.end();
            MRRR_CK(cudaGetLastError());
            size_t per = 2 * (size_t)nmax * sizeof(Y);
            // RQI in passes: two steps per eigenpair in the first pass (most
            // converge), then the parked ones, densely packed, in further
            // passes; the last pass has the rest of the max_rqi budget
            auto run_rqi = [&](int s0, int s1, cudaStream_t rs) -> int {
                if (s1 <= s0) return 0;
                const int S = s1 - s0;
                // persistent grid: enough warps for the list, at most the
                // tuned number of warps per SM, and within the scratch budget
                const size_t per_warp = 32 * per;
                long long G = ((long long)S + 31) / 32;
                int trial = -1;
                unsigned key = 0;
                int wps = kRqiTuneWarps[0];
                if (G > (long long)num_sms * kRqiTuneWarps[kRqiTuneCandidates - 1] &&
                    !(cfg.flags & MRRR_FLAG_NO_TUNE)) {
                    // only lists that can fill more than the smallest grid
                    // have anything to tune
                    auto lg = [](long long v) { unsigned b = 0; while (v > 1) { v >>= 1; ++b; } return b; };
                    key = (unsigned)sizeof(Y) << 16 | lg(S) << 8 | lg(nmax);
                    wps = rqi_tune_pick(key, &trial);
                }
                if (S > rqi_wps_list) {  // report the grid of the largest list
                    rqi_wps = wps;
                    rqi_wps_list = S;
                }
                G = std::min<long long>(G, (long long)num_sms * wps);
                G = std::min<long long>(G, std::max<long long>(1, (long long)(ScratchBudget<Y>::bytes() / per_warp)));
                Y* scratch = arena.alloc<Y>((size_t)G * 32 * 2 * nmax);
                int* park = arena.alloc<int>(2 * (size_t)S + 5);
                if (!scratch || !park) return MRRR_ERR_NOMEM;
                int* park_a = park;
                int* park_b = park + S;
                int* counts = park + 2 * (size_t)S;  // two park counters, three queue counters
                int* queues = counts + 2;
                if (cudaMemsetAsync(counts, 0, 5 * sizeof(int), rs) != cudaSuccess) return MRRR_ERR_CUDA;
                const int kPasses = 3;
                const int* list = single_list + s0;
                const int* total = nullptr;  // the first pass has all S items
                cudaEvent_t ta = nullptr, tb = nullptr;
                if (trial >= 0 && cudaEventCreate(&ta) == cudaSuccess && cudaEventCreate(&tb) == cudaSuccess)
                    cudaEventRecord(ta, rs);
                // no host synchronisation between passes: the stream (possibly
                // the side stream) keeps running while the host goes on
                for (int pass = 0; pass < kPasses; ++pass) {
                    bool final_pass = pass == kPasses - 1;
                    int* out = (pass % 2 == 0) ? park_a : park_b;
                    int* cnt = counts + (pass % 2);
                    int iters = pass == 0 ? 2 : (final_pass ? cfg.max_rqi : 3);
                    tl.begin(MRRR_PHASE_RQI, rs);
                    k_rqi<X, Y><<<(int)G, 32, 0, rs>>>(items, list, S, total, queues + pass, d_mats, d_blocks, cfg,
                                                        scratch, nmax, d_C, iters, final_pass ? 1 : 0, out, cnt);
                    tl.end(1, rs);
                    if (cudaGetLastError() != cudaSuccess) return MRRR_ERR_CUDA;
                    list = out;
                    total = cnt;
                }
                if (ta && tb) {
                    cudaEventRecord(tb, rs);
                    tune_runs.push_back({key, trial, ta, tb});
                }
                return 0;
            };
            // a4/a5: classification and the representation tree, level by level;
            // the singletons of the root level go to a second stream so their
            // RQI overlaps the (latency-bound) cluster levels
            const int* prev_members = nullptr;
            int nprev = K;
            int s_root = -1;
            for (int level = 0;; ++level) {
                Cluster* out = (level % 2 == 0) ? clus_a : clus_b;
                int* members = (level % 2 == 0) ? member_a : member_b;
                MRRR_CK(cudaMemsetAsync(&d_C->pool_need, 0, sizeof(unsigned long long), st));
                MRRR_CK(cudaMemsetAsync(&d_C->ncluster, 0, 2 * sizeof(int), st));  // ncluster, nmember
                bool force = level >= max_depth;
                double gt = force ? -INFINITY : cfg.gaptol;
                tl.begin(MRRR_PHASE_CLASSIFY);
                k_classify<<<grid_for(nprev), kThreads, 0, st>>>(items, prev_members, nprev, K, gt, single_list, out,
                                                                 members, d_C);
                tl.end();
                MRRR_CK(cudaGetLastError());
                if (int rc0 = from_device(ha, &C, d_C, 1, st)) return rc0;
                if (level == 0 && root_sep) {
                    // the root classification is all that was asked for
                    std::vector<Item> hitems(K);
                    if (int rc0 = from_device(ha, hitems.data(), items, (size_t)K, st)) return rc0;
                    root_sep->j.resize(K);
                    root_sep->matrix.resize(K);
                    root_sep->block.resize(K);
                    root_sep->rel.resize(K);
                    for (int t = 0; t < K; ++t) {
                        const Item& A = hitems[t];
                        root_sep->j[t] = A.j;
                        root_sep->matrix[t] = A.matrix;
                        root_sep->block[t] = A.block;
                        double rel = INFINITY;
                        if (t + 1 < K && hitems[t + 1].block == A.block) {
                            const Item& B = hitems[t + 1];
                            const double den = std::max(std::max(fabs(A.lo), fabs(A.hi)), std::max(fabs(B.lo), fabs(B.hi)));
                            rel = den > 0.0 ? (B.lo - A.hi) / den : 0.0;
                        }
                        root_sep->rel[t] = rel;
                    }
                    if (stats) tl.collect(stats);
                    return MRRR_OK;
                }
                if (level == 0) {
                    s_root = C.nsingle;
                    if (C.ncluster > 0 && s_root > 0) {
                        if (!side.start()) return MRRR_ERR_CUDA;
                        int rc = run_rqi(0, s_root, side.s);
                        if (rc) return rc;
                    } else {
                        s_root = 0;  // everything runs on the main stream below
                    }
                }
                if (C.ncluster == 0) break;
                MRRR_ALLOC(pool, Y, (size_t)C.pool_need);
                MRRR_ALLOC(pool_lo, Lo, (size_t)C.pool_need / 2);
                tl.begin(MRRR_PHASE_SHIFT);
                k_shift<Y, Lo><<<grid_for(C.ncluster, kLatThreads), kLatThreads, 0, st>>>(out, C.ncluster, items, d_blocks, pool,
                                                                          pool_lo, cfg, d_C);
                tl.end();
                MRRR_CK(cudaGetLastError());
                if (approximate(members, C.nmember, true, &d_C->qd_refine, MRRR_PHASE_REFINE)) return MRRR_ERR_CUDA;
                prev_members = members;
                nprev = C.nmember;
            }
            // a6/a7: RQI for the remaining singletons
            {
                int rc = run_rqi(s_root, C.nsingle, st);
                if (rc) return rc;
            }
            side.rejoin();
            // W ascending for matrices that split (see k_rank)
            tl.begin(MRRR_PHASE_FINISH);
            int fin_launches = 0;
            {
                std::vector<MatrixDesc> hm(P);
                if (int rc0 = from_device(ha, hm.data(), d_mats, (size_t)P, st)) return rc0;
                std::vector<int> sp;
                std::vector<long long> roff;
                long long rtot = 0;
                int maxk = 0;
                for (int p = 0; p < P; ++p) {
                    if (hm[p].nblocks > 1 && hm[p].kout > 1) {
                        sp.push_back(p);
                        roff.push_back(rtot);
                        rtot += hm[p].kout;
                        maxk = std::max(maxk, hm[p].kout);
                    }
                }
                if (!sp.empty()) {
                    const int ns = (int)sp.size();
                    MRRR_ALLOC(d_sp, int, ns);
                    MRRR_ALLOC(d_roff, long long, ns);
                    MRRR_ALLOC(d_rank, int, rtot);
                    MRRR_ALLOC(d_flag, int, ns);
                    if (int rc0 = to_device(ha, d_sp, sp.data(), (size_t)ns, st)) return rc0;
                    if (int rc0 = to_device(ha, d_roff, roff.data(), (size_t)ns, st)) return rc0;
                    MRRR_CK(cudaMemsetAsync(d_flag, 0, sizeof(int) * ns, st));
                    k_rank<X><<<dim3((maxk + kRankTile - 1) / kRankTile, ns), kRankTile, 0, st>>>(d_mats, d_sp, d_roff,
                                                                                                 d_rank, d_flag);
                    MRRR_CK(cudaGetLastError());
                    ++fin_launches;
                    std::vector<int> flag(ns);
                    if (int rc0 = from_device(ha, flag.data(), d_flag, (size_t)ns, st)) return rc0;
                    // the matrices that must be permuted, with their offsets
                    std::vector<int> fl;
                    std::vector<long long> froff, ftoff;
                    long long ttot = 0;
                    int maxkf = 0;
                    for (int q = 0; q < ns; ++q) {
                        if (!flag[q]) continue;
                        const MatrixDesc& M = hm[sp[q]];
                        fl.push_back(sp[q]);
                        froff.push_back(roff[q]);
                        ftoff.push_back(ttot);
                        ttot += (long long)M.n * M.kout;
                        maxkf = std::max(maxkf, M.kout);
                    }
                    if (!fl.empty()) {
                        const int nf = (int)fl.size();
                        MRRR_ALLOC(d_fl, int, nf);
                        MRRR_ALLOC(d_froff, long long, nf);
                        MRRR_ALLOC(d_ftoff, long long, nf);
                        MRRR_ALLOC(d_T, X, ttot);
                        MRRR_ALLOC(d_Wt, X, rtot);
                        if (int rc0 = to_device(ha, d_fl, fl.data(), (size_t)nf, st)) return rc0;
                        if (int rc0 = to_device(ha, d_froff, froff.data(), (size_t)nf, st)) return rc0;
                        if (int rc0 = to_device(ha, d_ftoff, ftoff.data(), (size_t)nf, st)) return rc0;
                        k_gather<X><<<dim3(maxkf, nf), 128, 0, st>>>(d_mats, d_fl, d_froff, d_rank, d_ftoff, d_T, d_Wt);
                        k_copy_back<X><<<dim3(maxkf, nf), 128, 0, st>>>(d_mats, d_fl, d_froff, d_ftoff, d_T, d_Wt);
                        MRRR_CK(cudaGetLastError());
                        fin_launches += 2;
                    }
                }
            }
            tl.end(fin_launches);
        }
    }
    if (int rc0 = from_device(ha, &C, d_C, 1, st)) return rc0;
    if (int rc0 = from_device(ha, mats, d_mats, (size_t)P, st)) return rc0;
    for (TuneRun& t : tune_runs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) rqi_tune_report(t.key, t.trial, ms);
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    int rc = 0;
    for (int p = 0; p < P && rc == 0; ++p) {
        if (mats[p].status == ST_ERR_NONFINITE) rc = MRRR_ERR_NONFINITE;
    }
    if (rc == 0 && C.noconv > 0) rc = MRRR_ERR_NOCONV;
    if (stats) {
        stats->nblocks = NB;
        stats->d_max = C.d_max;
        stats->nclusters = C.nclusters_total;
        stats->largest_cluster = C.largest_cluster;
        stats->reps_failed = C.reps_failed;
        stats->rqi_iters = C.rqi_iters;
        stats->fallbacks = C.fallbacks;
        stats->noconv = C.noconv;
        stats->qd_bisect = (long long)C.qd_bisect;
        stats->qd_refine = (long long)C.qd_refine;
        stats->qd_rqi = (long long)C.qd_rqi;
        stats->qd_shift = (long long)C.qd_shift;
        stats->qd_low = (long long)C.qd_steps_low;
        stats->verify_fail = C.verify_fail;
        stats->reps_relaxed = C.reps_relaxed;
        stats->rqi_warps_per_sm = rqi_wps;
        stats->rqi_rows = (long long)C.rqi_rows;
        stats->reps_backtracked = C.reps_backtracked;
        stats->reps_krr_relaxed = C.reps_krr_relaxed;
        {
            double k;
            memcpy(&k, &C.krr_max_bits, sizeof(k));
            stats->krr_max = k;
        }
        tl.collect(stats);
    }
    if (arena.failed) return MRRR_ERR_NOMEM;
    return rc;
}

}  // namespace mrrr
