// Device-tuned binary64 versions of the two hottest transforms: the Sturm
// count of the stationary qd transform (bisection and bracket checks) and the
// twisted factorization + solve of one RQI step.  They compute the same
// recurrences as negcount / twisted_solve in mrrr_core.cuh (see there for
// the formulas and the paper sections) with fewer FP64-pipe instructions:
//
//  * GB300 issues one FP64 instruction per SM sub-partition every ~64 cycles,
//    so every FP64 instruction on a recurrence is latency.  Sign tests, the
//    |gamma| comparison, zero tests and the arg-max are done on the IEEE bit
//    patterns with integer instructions instead of FP64 compares.
//  * The divide is a reciprocal estimate with Newton-Raphson refinement fused
//    into the next operation (see qdiv).
//  * Loads of the next row are issued one row ahead so memory latency
//    overlaps the FP64 chain.
#pragma once

#include "mrrr_core.cuh"

namespace mrrr {

#if defined(__CUDACC__)

__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
// 1 if x < 0 or x = -0 (sign bit), from the high word
__device__ __forceinline__ int dsign(double x) { return (int)((unsigned)__double2hiint(x) >> 31); }
// |x| as an unsigned integer with the same ordering as |x| (non-NaN)
__device__ __forceinline__ unsigned long long dabsbits(double x) {
    return (unsigned long long)dbits(x) & 0x7fffffffffffffffULL;
}
__device__ __forceinline__ bool dfinite(double x) { return ((unsigned)__double2hiint(x) & 0x7ff00000u) != 0x7ff00000u; }

// reciprocal estimate refined by `steps` Newton-Raphson iterations
template <int steps>
__device__ __forceinline__ double drcp(double b) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(b));
#pragma unroll
    for (int k = 0; k < steps; ++k) {
        double e = fma(-b, r, 1.0);
        r = fma(r, e, r);
    }
    return r;
}

// Sturm count (number of eigenvalues of L D L^T below tau) for bisection and
// bracket checks.  The reciprocal gets one Newton step (relative error
// ~2^-46): the count is exact for the rep perturbed element-wise by a few
// units of 2^-46, far inside what classification needs (relative accuracy
// 1e-2 gaptol >= 1e-12).  The loop runs unguarded; if a pivot vanished the
// recurrence produces a non-finite value and the guarded count is used.
__device__ __forceinline__ int negcount_fast(const double* __restrict__ D, const double* __restrict__ LLD, int n,
                                             double tau, double pivmin) {
    double s = -tau;
    int cnt = 0;
    double dn = __ldg(D), ln = __ldg(LLD);
    for (int i = 0; i < n - 1; ++i) {
        double di = dn, li = ln;
        dn = __ldg(D + i + 1);
        ln = __ldg(LLD + i + 1);
        double dp = di + s;
        cnt += dsign(dp);
        s = fma(s * li, drcp<1>(dp), -tau);
    }
    double dp = dn + s;
    cnt += dsign(dp);
    if (!dfinite(s) || !dfinite(dp)) return negcount<double>(D, LLD, n, tau, pivmin);
    return cnt;
}

// One twisted-factorization solve at lam for an eigenpair whose scratch
// arrays A, B (n words each) are contiguous; same results contract as
// twisted_solve: z in A (z_r = 1), returns r, inertia count and ||z||^2;
// *imax receives the index of the entry of largest magnitude.
__device__ __forceinline__ TwistResult<double> twisted_solve_fast(const double* __restrict__ rep, int n, double lam,
                                                                 double pivmin, double* __restrict__ A,
                                                                 double* __restrict__ B, double* gamma,
                                                                 int* imax) {
    const double* __restrict__ D = rep;
    const double* __restrict__ L = rep + n;
    const double* __restrict__ LD = rep + 2 * n;
    const double* __restrict__ LLD = rep + 3 * n;
    TwistResult<double> res;
    // stationary transform, top-down: l+_i -> A, s_i -> B
    double s = -lam;
    int neg = 0;
    bool bad = false;
    {
        double dn = __ldg(D), ldn = __ldg(LD), lnx = __ldg(L);
        for (int i = 0; i < n - 1; ++i) {
            double di = dn, ldi = ldn, li = lnx;
            dn = __ldg(D + i + 1);
            ldn = __ldg(LD + i + 1);
            lnx = __ldg(L + i + 1);
            double dp = di + s;
            neg += dsign(dp);
            double lp = ldi * drcp<2>(dp);
            A[i] = lp;
            B[i] = s;
            s = fma(lp * li, s, -lam);
        }
        double dp = dn + s;
        neg += dsign(dp);
        bad = !dfinite(s) || !dfinite(dp);
    }
    // progressive transform, bottom-up: gamma_k, u_k -> B
    double p = __ldg(D + n - 1) - lam;
    double gbest = s + p + lam;
    int r = n - 1;
    unsigned long long gb = dabsbits(gbest);
    {
        double lldn = n > 1 ? __ldg(LLD + n - 2) : 0.0, dn = n > 1 ? __ldg(D + n - 2) : 0.0;
        double lnx = n > 1 ? __ldg(L + n - 2) : 0.0, bn = n > 1 ? B[n - 2] : 0.0;
        for (int i = n - 2; i >= 0; --i) {
            double lldi = lldn, di = dn, li = lnx, si = bn;
            if (i > 0) {
                lldn = __ldg(LLD + i - 1);
                dn = __ldg(D + i - 1);
                lnx = __ldg(L + i - 1);
                bn = B[i - 1];
            }
            double om = lldi + p;
            double t = di * drcp<2>(om);
            double um = li * t;
            p = fma(p, t, -lam);
            double g = (si + p) + lam;
            B[i] = um;
            unsigned long long ga = dabsbits(g);
            if (ga <= gb) {  // smallest index on ties
                gb = ga;
                gbest = g;
                r = i;
            }
        }
        bad = bad || !dfinite(p);
    }
    if (bad) {
        // a pivot vanished: redo with the guarded generic transform
        Scratch<double> W;
        W.a = A;
        W.b = B;
        W.stride = 1;
        res = twisted_solve<double>(rep, n, lam, pivmin, W, gamma);
        unsigned long long zb = 0;
        int im = 0;
        for (int i = 0; i < n; ++i) {
            unsigned long long a = dabsbits(A[i]);
            if (a > zb) {
                zb = a;
                im = i;
            }
        }
        *imax = im;
        return res;
    }
    // N_r^T z = e_r: every lane runs n-1 steps -- first r steps downward from
    // r (z_i = -l+_i z_{i+1}), then n-1-r steps upward (z_{i+1} = -u_i z_i)
    // -- so lanes with different r do not diverge.  The coefficient of the
    // next step is loaded one step ahead.
    double nrm2 = 1.0;
    A[r] = 1.0;
    unsigned long long zmax = dabsbits(1.0);
    int im = r;
    double zprev = 1.0;   // z at the previous position of the walk
    double zprev2 = 0.0;  // z two positions back (for the zero rule)
    double cn = n > 1 ? (0 < r ? A[r - 1] : B[0]) : 0.0;
    for (int k = 0; k < n - 1; ++k) {
        double c = cn;
        if (k + 1 < n - 1) cn = (k + 1 < r) ? A[r - 2 - k] : B[k + 1];
        int i;
        bool down = k < r;
        if (down) {
            i = r - 1 - k;
        } else {
            i = k + 1;
            if (k == r) {  // the upward walk restarts at z_r = 1
                zprev = 1.0;
                zprev2 = 0.0;
            }
        }
        double z;
        if (dabsbits(zprev) != 0) {
            z = -(c * zprev);
        } else if (down) {
            // row i+1 with z_{i+1} = 0: e_i z_i + e_{i+1} z_{i+2} = 0
            z = (i + 2 < n) ? -(__ldg(LD + i + 1) / __ldg(LD + i)) * zprev2 : 0.0;
        } else {
            // row i-1 with z_{i-1} = 0: e_{i-2} z_{i-2} + e_{i-1} z_i = 0
            z = (i >= 2) ? -(__ldg(LD + i - 2) / __ldg(LD + i - 1)) * zprev2 : 0.0;
        }
        A[i] = z;
        nrm2 = fma(z, z, nrm2);
        unsigned long long za = dabsbits(z);
        if (za > zmax || (za == zmax && i < im)) {
            zmax = za;
            im = i;
        }
        zprev2 = zprev;
        zprev = z;
    }
    *imax = im;
    res.r = r;
    res.neg = neg;
    res.nrm2 = nrm2;
    *gamma = gbest;
    return res;
}

#endif  // __CUDACC__

}  // namespace mrrr
