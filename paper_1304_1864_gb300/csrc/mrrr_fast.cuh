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

// rows per software-prefetch group for the per-eigenpair scratch arrays
constexpr int kG = 8;
// bit pattern of 2^-900: entries of z (z_r = 1) below it are the underflowed
// tail of the vector
constexpr unsigned long long kZTinyBits = (unsigned long long)(1023 - 900) << 52;

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
// Guarded fallbacks, kept out of line so that they do not weigh on the
// register allocation and scheduling of the unguarded hot loops.
static __device__ __noinline__ int negcount_guarded(const double* D, const double* LLD, int n, double tau, double pivmin) {
    return negcount<double>(D, LLD, n, tau, pivmin);
}

__device__ __forceinline__ int negcount_fast(const double* __restrict__ D, const double* __restrict__ LLD, int n,
                                             double tau, double pivmin) {
    double s = -tau;
    int cnt = 0;
    int i = 0;
    // four rows per iteration with their loads issued together
    for (; i + 4 <= n - 1; i += 4) {
        const int ip = min(i + kPrefetch, n - 1);
        pf_l2(D + ip);
        pf_l2(LLD + ip);
        double d0 = __ldg(D + i), d1 = __ldg(D + i + 1), d2 = __ldg(D + i + 2), d3 = __ldg(D + i + 3);
        double l0 = __ldg(LLD + i), l1 = __ldg(LLD + i + 1), l2 = __ldg(LLD + i + 2), l3 = __ldg(LLD + i + 3);
        double dp = d0 + s;
        cnt += dsign(dp);
        s = fma(s * l0, drcp<1>(dp), -tau);
        dp = d1 + s;
        cnt += dsign(dp);
        s = fma(s * l1, drcp<1>(dp), -tau);
        dp = d2 + s;
        cnt += dsign(dp);
        s = fma(s * l2, drcp<1>(dp), -tau);
        dp = d3 + s;
        cnt += dsign(dp);
        s = fma(s * l3, drcp<1>(dp), -tau);
    }
    for (; i < n - 1; ++i) {
        double dp = __ldg(D + i) + s;
        cnt += dsign(dp);
        s = fma(s * __ldg(LLD + i), drcp<1>(dp), -tau);
    }
    double dp = __ldg(D + n - 1) + s;
    cnt += dsign(dp);
    if (!dfinite(s) || !dfinite(dp)) return negcount_guarded(D, LLD, n, tau, pivmin);
    return cnt;
}

// Stationary transform on rows [0, m): l+_i -> A[i] and, if B != nullptr,
// s_i -> B[i].  Returns s_m; *neg += number of negative d+_i, i < m.
__device__ __forceinline__ double stationary_fast(const double* __restrict__ D, const double* __restrict__ L,
                                                  const double* __restrict__ LD, int m, double lam,
                                                  double* __restrict__ A, double* __restrict__ B, int* neg) {
    double s = -lam;
    if (m <= 0) return s;
    int c = 0;
    double dn = __ldg(D), ldn = __ldg(LD), lnx = __ldg(L);
    for (int i = 0; i < m; ++i) {
        const int ip = min(i + kPrefetch, m);
        pf_l2(D + ip);
        pf_l2(LD + ip);
        pf_l2(L + ip);
        double di = dn, ldi = ldn, li = lnx;
        dn = __ldg(D + i + 1);
        ldn = __ldg(LD + i + 1);
        lnx = __ldg(L + i + 1);
        double dp = di + s;
        c += dsign(dp);
        double lp = ldi * drcp<2>(dp);
        A[i] = lp;
        if (B) B[i] = s;
        s = fma(lp * li, s, -lam);
    }
    *neg += c;
    return s;
}

static __device__ __noinline__ double dstqds_guarded(const double* parent, int n, double tau, double pivmin, double* out,
                                             float* out_lo) {
    double g = dstqds<double>(parent, n, tau, pivmin, out);
    if (out && g < INFINITY) {
        for (int i = 0; i < n; ++i) {
            out_lo[i] = (float)out[i];
            out_lo[n + i] = (float)out[3 * n + i];
        }
    }
    return g;
}

// Child representation parent - tau I (stationary transform, as dstqds) with
// the element growth max |d+_i| tracked on the bit patterns; if out != null
// the child rep is written there and its rounded copy [D | LLD] to out_lo,
// in the same pass.  Unguarded; a vanished pivot makes the result
// non-finite and the guarded generic transform is used instead.
__device__ __forceinline__ double dstqds_fast(const double* __restrict__ parent, int n, double tau, double pivmin,
                                              double* __restrict__ out, float* __restrict__ out_lo) {
    const double* __restrict__ D = parent;
    const double* __restrict__ L = parent + n;
    const double* __restrict__ LD = parent + 2 * n;
    double s = -tau;
    unsigned long long gmax = 0;
    double dn = __ldg(D), ldn = __ldg(LD), lnx = __ldg(L);
    for (int i = 0; i < n - 1; ++i) {
        double di = dn, ldi = ldn, li = lnx;
        dn = __ldg(D + i + 1);
        ldn = __ldg(LD + i + 1);
        lnx = __ldg(L + i + 1);
        double dp = di + s;
        unsigned long long a = dabsbits(dp);
        gmax = a > gmax ? a : gmax;
        double lp = ldi * drcp<2>(dp);
        s = fma(lp * li, s, -tau);
        if (out) {
            double ldp = dp * lp;
            double lldp = ldp * lp;
            out[i] = dp;
            out[n + i] = lp;
            out[2 * n + i] = ldp;
            out[3 * n + i] = lldp;
            out_lo[i] = (float)dp;
            out_lo[n + i] = (float)lldp;
        }
    }
    double dp = dn + s;
    unsigned long long a = dabsbits(dp);
    gmax = a > gmax ? a : gmax;
    if (!dfinite(s) || !dfinite(dp) || gmax >= 0x7ff0000000000000ULL)
        return dstqds_guarded(parent, n, tau, pivmin, out, out_lo);
    if (out) {
        out[n - 1] = dp;
        out[2 * n - 1] = 0.0;
        out[3 * n - 1] = 0.0;
        out[4 * n - 1] = 0.0;
        out_lo[n - 1] = (float)dp;
        out_lo[2 * n - 1] = 0.0f;
    }
    return __longlong_as_double((long long)gmax);
}

// N_r^T z = e_r from l+ (A, rows < r) and u (B, rows >= r); z overwrites A.
// Every lane runs n-1 steps -- first r steps downward from r (z_i = -l+_i
// z_{i+1}), then n-1-r steps upward (z_{i+1} = -u_i z_i) -- so lanes with
// different r do not diverge.  The common step is written with selects
// instead of branches (the row index, the restart at r, the arg-max); only
// a zero entry takes the zero rule.  The coefficients are loaded a group of
// kG steps ahead.  Returns ||z||^2; *imax = index of the largest |z_i|
// (smallest index on ties).
__device__ __forceinline__ double solve_twisted_fast(const double* __restrict__ LD, int n, int r,
                                                     double* __restrict__ A, const double* __restrict__ B,
                                                     int* imax) {
    double nrm2 = 1.0;
    A[r] = 1.0;
    unsigned long long zmax = dabsbits(1.0);
    int im = r;
    double zprev = 1.0;   // z at the previous position of the walk
    double zprev2 = 0.0;  // z two positions back (for the zero rule)
    const int steps = n - 1;
    // coefficient of walk step k: l+_{r-1-k} downward, u_k upward
    double cur[kG], nxt[kG];
#pragma unroll
    for (int k = 0; k < kG; ++k) {
        const double* pp = k < r ? A + (r - 1 - k) : B + k;
        cur[k] = k < steps ? *pp : 0.0;
    }
    for (int k0 = 0; k0 < steps; k0 += kG) {
        {
            const int kp = min(k0 + kPrefetch, steps - 1);
            pf_l2(kp < r ? A + (r - 1 - kp) : B + kp);
        }
#pragma unroll
        for (int q = 0; q < kG; ++q) {
            const int kk = k0 + kG + q;
            const double* pp = kk < r ? A + (r - 1 - kk) : B + kk;
            nxt[q] = kk < steps ? *pp : 0.0;
        }
#pragma unroll
        for (int q = 0; q < kG; ++q) {
            const int k = k0 + q;
            if (k < steps) {
                const bool down = k < r;
                const int i = down ? r - 1 - k : k + 1;
                const bool reset = k == r;  // the upward walk restarts at z_r = 1
                zprev = reset ? 1.0 : zprev;
                zprev2 = reset ? 0.0 : zprev2;
                double z = -(cur[q] * zprev);
                if (dabsbits(zprev) == 0) {
                    if (dabsbits(zprev2) < kZTinyBits) {
                        // a zero next to a zero or a value below 2^-900 (z_r =
                        // 1): the underflowed tail of a localized vector,
                        // which stays zero from here on (without this the
                        // rule below would revive subnormals every other row)
                        z = 0.0;
                    } else if (down) {
                        // row i+1 with z_{i+1} = 0: e_i z_i + e_{i+1} z_{i+2} = 0
                        // (the quotient by the transforms' reciprocal, not an
                        // IEEE divide: localized vectors take this rule often)
                        z = (i + 2 < n) ? -(__ldg(LD + i + 1) * drcp<2>(__ldg(LD + i))) * zprev2 : 0.0;
                    } else {
                        // row i-1 with z_{i-1} = 0: e_{i-2} z_{i-2} + e_{i-1} z_i = 0
                        z = (i >= 2) ? -(__ldg(LD + i - 2) * drcp<2>(__ldg(LD + i - 1))) * zprev2 : 0.0;
                    }
                }
                A[i] = z;
                nrm2 = fma(z, z, nrm2);
                const unsigned long long za = dabsbits(z);
                const bool better = za > zmax || (za == zmax && i < im);
                zmax = better ? za : zmax;
                im = better ? i : im;
                zprev2 = zprev;
                zprev = z;
            }
        }
#pragma unroll
        for (int q = 0; q < kG; ++q) cur[q] = nxt[q];
    }
    *imax = im;
    return nrm2;
}

// Guarded generic twisted solve (out of line), with the arg-max of |z|.
static __device__ __noinline__ TwistResult<double> twisted_guarded(const double* rep, int n, double lam, double pivmin,
                                                            double* A, double* B, double* gamma, int* imax) {
    Scratch<double> W;
    W.a = A;
    W.b = B;
    W.stride = 1;
    TwistResult<double> res = twisted_solve<double>(rep, n, lam, pivmin, W, gamma);
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

// One twisted-factorization solve at lam for an eigenpair whose scratch
// arrays A, B (n words each) are contiguous; same results contract as
// twisted_solve: z in A (z_r = 1), returns r, inertia count and ||z||^2;
// *imax receives the index of the entry of largest magnitude.
//
// r_fixed < 0: the full factorization -- stationary transform top-down,
// progressive transform bottom-up, r = argmin |gamma_k| (Sec. 2, RQI steps
// (i)-(ii)).  r_fixed >= 0: the twist index is given (the largest entry of
// the previous iterate, as e_r then has a large component along the wanted
// eigenvector), and only rows < r of the stationary and rows > r of the
// progressive transform are needed -- one pass instead of two.  In both
// cases the inertia of Delta_r = diag(d+_0..d+_{r-1}, gamma_r,
// w_{r+1}..w_{n-1}) is the Sturm count at lam (Sylvester), used to update
// the bisection bracket.
__device__ __forceinline__ TwistResult<double> twisted_solve_fast(const double* __restrict__ rep, int n, double lam,
                                                                 double pivmin, double* __restrict__ A,
                                                                 double* __restrict__ B, double* gamma, int* imax,
                                                                 int r_fixed = -1) {
    const double* __restrict__ D = rep;
    const double* __restrict__ L = rep + n;
    const double* __restrict__ LD = rep + 2 * n;
    const double* __restrict__ LLD = rep + 3 * n;
    TwistResult<double> res;
    int neg = 0;
    int r;
    double gbest;
    bool bad;
    if (r_fixed < 0) {
        // stationary transform, top-down: l+_i -> A, s_i -> B
        double s = stationary_fast(D, L, LD, n - 1, lam, A, B, &neg);
        double dlast = __ldg(D + n - 1) + s;
        neg += dsign(dlast);
        bad = !dfinite(s) || !dfinite(dlast);
        // progressive transform, bottom-up: gamma_k, u_k -> B
        double p = __ldg(D + n - 1) - lam;
        gbest = s + p + lam;
        r = n - 1;
        unsigned long long gb = dabsbits(gbest);
        // rows n-2 .. 0 in groups of kG; the s_i of the next group (per-lane
        // scratch, usually not in L1) are loaded a whole group ahead
        double cur[kG], nxt[kG];
#pragma unroll
        for (int k = 0; k < kG; ++k) cur[k] = (n - 2 - k >= 0) ? B[n - 2 - k] : 0.0;
        for (int i0 = n - 2; i0 >= 0; i0 -= kG) {
            {
                const int ip = max(i0 - kPrefetch, 0);
                pf_l2(LLD + ip);
                pf_l2(D + ip);
                pf_l2(L + ip);
                pf_l2(B + ip);
            }
#pragma unroll
            for (int k = 0; k < kG; ++k) {
                int ii = i0 - kG - k;
                nxt[k] = ii >= 0 ? B[ii] : 0.0;
            }
#pragma unroll
            for (int k = 0; k < kG; ++k) {
                int i = i0 - k;
                if (i >= 0) {
                    double om = __ldg(LLD + i) + p;
                    double t = __ldg(D + i) * drcp<2>(om);
                    double um = __ldg(L + i) * t;
                    p = fma(p, t, -lam);
                    double g = (cur[k] + p) + lam;
                    B[i] = um;
                    unsigned long long ga = dabsbits(g);
                    if (ga <= gb) {  // smallest index on ties
                        gb = ga;
                        gbest = g;
                        r = i;
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < kG; ++k) cur[k] = nxt[k];
        }
        bad = bad || !dfinite(p);
    } else {
        // fixed r: rows < r of the stationary transform (l+ -> A) and rows
        // > r of the progressive one (u -> B, counting the signs of the
        // pivots w_{i+1}), as one walk of n-1 steps per lane -- r stationary
        // rows top-down, then n-1-r progressive rows bottom-up -- so lanes
        // with different r do not diverge.  Both rows have the form
        // q = 1 / (a + x), m = b q, with (a, b) = (d_i, ld_i) and the update
        // x = x (m l_i) - lam for the stationary row, (a, b) = (lld_i, d_i)
        // and x = x m - lam for the progressive one.
        r = r_fixed;
        const double dlast = __ldg(D + n - 1) - lam;
        double x = -lam, s_r = 0.0;
        if (r == 0) {
            s_r = x;
            x = dlast;
        }
        bool st = 0 < r;
        int i = st ? 0 : n - 2;
        double a = __ldg((st ? D : LLD) + i), b = __ldg((st ? LD : D) + i), l = __ldg(L + i);
        for (int k = 0; k < n - 1; ++k) {
            const int ic = i;
            const bool stc = st;
            const double ac = a, bc = b, lc = l;
            // operands of the next step, one step ahead; their lines
            // kPrefetch steps ahead into L2
            {
                const int kp = min(k + kPrefetch, n - 2);
                const bool sp = kp < r;
                const int ipf = sp ? kp : n - 2 - (kp - r);
                pf_l2((sp ? D : LLD) + ipf);
                pf_l2((sp ? LD : D) + ipf);
                pf_l2(L + ipf);
            }
            const int k1 = k + 1;
            st = k1 < r;
            i = st ? k1 : n - 2 - (k1 - r);
            if (k1 < n - 1) {
                a = __ldg((st ? D : LLD) + i);
                b = __ldg((st ? LD : D) + i);
                l = __ldg(L + i);
            }
            const double den = ac + x;
            neg += dsign(den);
            const double m = bc * drcp<2>(den);
            const double ml = m * lc;
            *((stc ? A : B) + ic) = stc ? m : ml;
            x = fma(x, stc ? ml : m, -lam);
            if (k1 == r) {
                s_r = x;
                x = dlast;
            }
        }
        // the switch after row r-1 has run for every r >= 1 (for r = n-1 at
        // the last step, leaving p_{n-1} = d_{n-1} - lam)
        const double p = x;
        gbest = s_r + p + lam;
        neg += dsign(gbest);
        bad = !dfinite(s_r) || !dfinite(p) || !dfinite(gbest);
    }
    if (bad) return twisted_guarded(rep, n, lam, pivmin, A, B, gamma, imax);
    res.nrm2 = solve_twisted_fast(LD, n, r, A, B, imax);
    res.r = r;
    res.neg = neg;
    *gamma = gbest;
    return res;
}

// L D L^T factorization of T - mu I for the root representation (as
// ldl_factor): d_0 = a_0 - mu, l_i = b_i / d_i, d_{i+1} = (a_{i+1} - mu) -
// l_i b_i.  The chain from d_i to d_{i+1} is the reciprocal (two Newton
// steps) and one FMA with b_i^2 formed off the chain; the definiteness and
// finiteness tests and max |d_i| run on the bit patterns.  Returns max |d_i|,
// or +inf if a pivot has the wrong sign, vanished or overflowed.
__device__ __forceinline__ double ldl_factor_fast(const double* __restrict__ a, const double* __restrict__ b, int n,
                                                  double mu, int sgn, double* __restrict__ rep) {
    double* D = rep;
    double* L = rep + n;
    const int want = sgn < 0 ? 1 : 0;  // sign bit every pivot must have
    double d = a[0] - mu;
    unsigned long long gmax = 0;
    bool bad = false;
    double an = n > 1 ? a[1] : 0.0, bn = b[0];
    for (int i = 0; i < n - 1; ++i) {
        double ai1 = an, bi = bn;
        if (i + 2 < n) an = a[i + 2];
        if (i + 1 < n - 1) bn = b[i + 1];
        unsigned long long ab = dabsbits(d);
        bad |= (dsign(d) != want) | (ab == 0ULL) | !dfinite(d);
        gmax = ab > gmax ? ab : gmax;
        D[i] = d;
        double r = drcp<2>(d);
        L[i] = bi * r;
        d = fma(-(bi * bi), r, ai1 - mu);
    }
    unsigned long long ab = dabsbits(d);
    bad |= (dsign(d) != want) | (ab == 0ULL) | !dfinite(d);
    gmax = ab > gmax ? ab : gmax;
    D[n - 1] = d;
    L[n - 1] = 0.0;
    return bad ? INFINITY : __longlong_as_double((long long)gmax);
}

#endif  // __CUDACC__

}  // namespace mrrr
