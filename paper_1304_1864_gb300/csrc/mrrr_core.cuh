// Per-item building blocks of MRRR (Algorithm 1), written once for every
// working precision Y in {float, double, dd} and usable from host or device.
//
// A representation ("rep") of a tridiagonal is the lower bidiagonal
// factorization L D L^T in N-representation (d_1..d_n, l_1..l_{n-1}; Sec. 2,
// "Choice of representations" -- the form the paper's own solvers use,
// Sec. 4.1), stored contiguously in working precision together with the
// derived data LD_i = d_i l_i and LLD_i = d_i l_i^2:
//
//     rep[0 .. n)    D
//     rep[n .. 2n)   L      (entry n-1 unused)
//     rep[2n .. 3n)  LD     (entry n-1 unused)
//     rep[3n .. 4n)  LLD    (entry n-1 unused)
//
// The qd transforms below are the differential stationary and progressive
// transforms of Dhillon and Parlett, which the paper relies on for the
// element-wise mixed relatively stable shift M - tau I (Sec. 2, "Shifting the
// spectrum") and for the twisted factorizations of the Rayleigh quotient
// iteration (Sec. 2, "Rayleigh quotient iteration"):
//
//   stationary (L D L^T - tau I = L+ D+ L+^T):
//       s_1 = -tau;  d+_i = d_i + s_i;  l+_i = d_i l_i / d+_i;
//       s_{i+1} = l+_i l_i s_i - tau = LLD_i s_i / d+_i - tau;  d+_n = d_n + s_n
//   progressive (L D L^T - tau I = U W U^T, bottom to top):
//       p_n = d_n - tau;  w_{i+1} = LLD_i + p_{i+1};  t = d_i / w_{i+1};
//       u_i = l_i t;  p_i = p_{i+1} t - tau
//   twisted factorization at index k: gamma_k = s_k + p_k + tau
//       (n = 1: gamma_1 = d_1 - tau), and N_r^T z = e_r gives
//       z_r = 1, z_i = -l+_i z_{i+1} (i < r), z_{i+1} = -u_i z_i (i >= r).
#pragma once

#include <cfloat>
#include <cmath>
#include <cstdint>

#include "mrrr_dd.cuh"

namespace mrrr {

// ------------------------------------------------------------ precision

template <class Y> struct Prec;
template <> struct Prec<float> {
    static constexpr double eps = 5.9604644775390625e-08;   // 2^-24 (Table 1)
    static constexpr double tiny = 1.1754943508222875e-38;  // smallest normal
};
template <> struct Prec<double> {
    static constexpr double eps = 1.1102230246251565e-16;   // 2^-53 (Table 1)
    static constexpr double tiny = 2.2250738585072014e-308;
};
template <> struct Prec<dd> {
    static constexpr double eps = 4.930380657631324e-32;    // 2^-104 (conservative)
    static constexpr double tiny = 2.2250738585072014e-308;
};

MRRR_HD double to_d(float x) { return (double)x; }
MRRR_HD double to_d(double x) { return x; }
MRRR_HD double to_d(const dd& x) { return x.hi + x.lo; }

template <class Y> MRRR_HD Y from_d(double x);
template <> MRRR_HD float from_d<float>(double x) { return (float)x; }
template <> MRRR_HD double from_d<double>(double x) { return x; }
template <> MRRR_HD dd from_d<dd>(double x) { return dd(x); }

MRRR_HD float yabs(float x) { return fabsf(x); }
MRRR_HD double yabs(double x) { return fabs(x); }
MRRR_HD dd yabs(const dd& x) { return dd_abs(x); }

MRRR_HD bool yneg(float x) { return x < 0.0f; }
MRRR_HD bool yneg(double x) { return x < 0.0; }
MRRR_HD bool yneg(const dd& x) { return x.hi < 0.0; }

MRRR_HD bool yfinite(float x) { return isfinite(x); }
MRRR_HD bool yfinite(double x) { return isfinite(x); }
MRRR_HD bool yfinite(const dd& x) { return dd_isfinite(x); }

MRRR_HD float ysqrt(float x) { return sqrtf(x); }
MRRR_HD double ysqrt(double x) { return sqrt(x); }
MRRR_HD dd ysqrt(const dd& x) { return dd_sqrt(x); }

// |a| < b for the pivot guard
template <class Y> MRRR_HD bool ysmall(const Y& a, const Y& b) { return yabs(a) < b; }

// ------------------------------------------------------------ division in the qd transforms

// Quotient used by every qd transform.  In binary64 on the GPU it is a * r
// with r = 1/b from the hardware estimate (rcp.approx.ftz.f64, about 23
// bits) refined by two Newton-Raphson steps r <- r + r (1 - b r), the
// classical iteration for the reciprocal (each step squares the relative
// error).  The quotient is within a few units in the last place of a/b -- a
// constant factor in the element-wise relative error bounds the qd
// transforms are analysed with -- and its dependent chain is ~40 % shorter
// than the correctly rounded division (FP64 runs at 1/64 of the FP32 rate
// on this GPU, so every FP64 instruction on a recurrence counts).  Pivots
// are kept at |b| >= pivmin >= 4 * DBL_MIN, so b is never subnormal.
template <class Y> MRRR_HD Y qdiv(const Y& a, const Y& b) { return a / b; }
template <> MRRR_HD double qdiv<double>(const double& a, const double& b) {
#if defined(__CUDA_ARCH__)
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(b));
    double e = fma(-b, r, 1.0);
    r = fma(r, e, r);
    e = fma(-b, r, 1.0);
    r = fma(r, e, r);
    return a * r;
#else
    return a / b;
#endif
}

// Fast binary32 quotient for the low-precision pre-bisection only (its
// counts are always re-checked in the working precision).
MRRR_HD float fdiv_lo(float a, float b) {
#if defined(__CUDA_ARCH__)
    return __fdividef(a, b);
#else
    return a / b;
#endif
}
MRRR_HD double fdiv_lo(double a, double b) { return qdiv<double>(a, b); }

// Software prefetch into L2 for the row loops.  A lane streams through its
// own representation (a child rep of a cluster, or the scratch of its
// eigenpair) one row per step, and each row is one dependent chain of
// FP64 latency long; loading only the next row leaves DRAM latency exposed
// whenever the rep is not cache resident.  The loops therefore ask for the
// line kPrefetch rows ahead (a line holds 16 binary64 / 32 binary32 values;
// the caller keeps the row inside the array).  No register is tied up and
// the host build ignores it.
constexpr int kPrefetch = 64;
MRRR_HD void pf_l2(const void* p) {
#if defined(__CUDA_ARCH__)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
#else
    (void)p;
#endif
}

// ------------------------------------------------------------ random perturbation

// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) as a counter-based generator:
// the value for counter c is the finaliser applied to seed + (c+1)*golden.
MRRR_HD uint64_t splitmix64_at(uint64_t seed, uint64_t c) {
    uint64_t z = seed + (c + 1ULL) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// uniform in [-1, 1) with 53 random bits
MRRR_HD double sym_uniform(uint64_t seed, uint64_t c) {
    return (double)(splitmix64_at(seed, c) >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// ------------------------------------------------------------ rep access

template <class Y> struct RepPtr {
    const Y* D;
    const Y* L;
    const Y* LD;
    const Y* LLD;
    MRRR_HD RepPtr(const Y* base, int n) : D(base), L(base + n), LD(base + 2 * n), LLD(base + 3 * n) {}
};

// ------------------------------------------------------------ negcount

// Number of eigenvalues of the rep (L D L^T) strictly below tau: the count of
// negative pivots d+_i of the stationary transform (Sylvester's law of
// inertia).  A pivot with |d+_i| < pivmin is replaced by -pivmin.
template <class Y>
MRRR_HD int negcount(const Y* __restrict__ D, const Y* __restrict__ LLD, int n, Y tau, Y pivmin) {
    Y s = -tau;
    int cnt = 0;
    for (int i = 0; i < n - 1; ++i) {
        Y dp = D[i] + s;
        if (ysmall(dp, pivmin)) dp = -pivmin;
        cnt += yneg(dp) ? 1 : 0;
        s = qdiv<Y>(s * LLD[i], dp) - tau;
    }
    Y dp = D[n - 1] + s;
    if (ysmall(dp, pivmin)) dp = -pivmin;
    cnt += yneg(dp) ? 1 : 0;
    return cnt;
}

// The same count in a low precision Lo (binary32 under a binary64 working
// precision, binary64 under double-double) on a rounded copy of the rep:
// the pre-bisection of Sec. 3.2 ("Arithmetic used to approximate
// eigenvalues"), whose brackets are then verified in the working precision.
template <class Lo>
MRRR_HD int negcount_lo(const Lo* __restrict__ D, const Lo* __restrict__ LLD, int n, Lo tau, Lo pivmin) {
    Lo s = -tau;
    int cnt = 0;
    for (int i = 0; i < n - 1; ++i) {
        const int ip = min(i + kPrefetch, n - 1);
        pf_l2(D + ip);
        pf_l2(LLD + ip);
        Lo dp = D[i] + s;
        if (!(fabs(dp) >= pivmin)) dp = -pivmin;  // also catches NaN
        cnt += dp < Lo(0) ? 1 : 0;
        s = fdiv_lo(s * LLD[i], dp) - tau;
    }
    Lo dp = D[n - 1] + s;
    if (!(fabs(dp) >= pivmin)) dp = -pivmin;
    cnt += dp < Lo(0) ? 1 : 0;
    return cnt;
}

// Twist index for the first RQI step from the rounded low-precision copy
// [D | LLD] of the representation: gamma_k = s_k + p_k + tau from the
// stationary (s) and progressive (p) transforms at tau, r = argmin |gamma_k|
// (Sec. 2, the twisted factorization's choice of r), in the low precision.
// Only the index comes from here; the step itself -- gamma_r, the inertia
// and the vector -- runs in the working precision at that r, and any r at
// which the wanted eigenvector has a large entry serves.  s_store holds n
// values of scratch.  Returns -1 if the sweep met a vanished pivot or an
// overflow (the caller then factors fully in the working precision).
template <class Lo>
MRRR_HD int twist_index_lo(const Lo* __restrict__ D, const Lo* __restrict__ LLD, int n, Lo tau,
                           Lo* __restrict__ s_store) {
    Lo s = -tau;
    for (int i = 0; i < n - 1; ++i) {
        const int ip = min(i + kPrefetch, n - 1);
        pf_l2(D + ip);
        pf_l2(LLD + ip);
        s_store[i] = s;
        s = fdiv_lo(s * LLD[i], D[i] + s) - tau;
    }
    Lo p = D[n - 1] - tau;
    Lo gbest = s + p + tau;
    int r = n - 1;
    for (int i = n - 2; i >= 0; --i) {
        const int ip = max(i - kPrefetch, 0);
        pf_l2(D + ip);
        pf_l2(LLD + ip);
        pf_l2(s_store + ip);
        p = fdiv_lo(D[i] * p, LLD[i] + p) - tau;
        Lo g = s_store[i] + p + tau;
        if (fabs(g) <= fabs(gbest)) {  // smallest index on ties
            gbest = g;
            r = i;
        }
    }
    if (!isfinite(gbest) || !isfinite(p) || !isfinite(s)) return -1;
    return r;
}

// ------------------------------------------------------------ root representation

// L D L^T factorization of (T - mu I) in working precision for the rows
// a[0..n), b[0..n-1) (diagonal, off-diagonal; already scaled).  Writes D and
// L into rep (rep layout above) and returns max |d_i|, or +inf if a pivot
// vanished / the factorization is not definite with the sign `sgn`.
template <class Y>
MRRR_HD double ldl_factor(const double* a, const double* b, int n, double mu, int sgn, Y* rep) {
    Y* D = rep;
    Y* L = rep + n;
    Y d = from_d<Y>(a[0]) - from_d<Y>(mu);
    double growth = 0.0;
    for (int i = 0; i < n; ++i) {
        if (i > 0) {
            // d_{i} = (a_i - mu) - l_{i-1} e_{i-1}
            d = (from_d<Y>(a[i]) - from_d<Y>(mu)) - L[i - 1] * from_d<Y>(b[i - 1]);
        }
        double dv = to_d(d);
        if (!(dv * sgn > 0.0) || !isfinite(dv)) return INFINITY;
        D[i] = d;
        growth = fmax(growth, fabs(dv));
        if (i < n - 1) L[i] = qdiv<Y>(from_d<Y>(b[i]), d);
    }
    L[n - 1] = from_d<Y>(0.0);
    return growth;
}

// Multiply every d_i and l_i by (1 + xi * r) with r uniform in [-1, 1) from
// the counter-based generator (Algorithm 1, line 2; Sec. 3.2, "Random
// perturbations"), then form LD and LLD.
template <class Y>
MRRR_HD void perturb_and_derive(Y* rep, int n, double xi, uint64_t seed, uint64_t counter0) {
    Y* D = rep;
    Y* L = rep + n;
    Y* LD = rep + 2 * n;
    Y* LLD = rep + 3 * n;
    for (int i = 0; i < n; ++i) {
        if (xi > 0.0) {
            double rd = xi * sym_uniform(seed, counter0 + 2ULL * (uint64_t)i);
            D[i] = D[i] + D[i] * from_d<Y>(rd);
            if (i < n - 1) {
                double rl = xi * sym_uniform(seed, counter0 + 2ULL * (uint64_t)i + 1ULL);
                L[i] = L[i] + L[i] * from_d<Y>(rl);
            }
        }
    }
    for (int i = 0; i < n - 1; ++i) {
        LD[i] = D[i] * L[i];
        LLD[i] = LD[i] * L[i];
    }
    LD[n - 1] = from_d<Y>(0.0);
    LLD[n - 1] = from_d<Y>(0.0);
}

// ------------------------------------------------------------ shifted child rep

// Stationary transform of the parent rep at shift tau.  If `out` is non-NULL
// the child rep (D+, L+, LD+, LLD+) is written there.  Returns the element
// growth max |d+_i|, or +inf if a non-finite value appeared.  With erep the
// child is kept in e-representation (Sec. 3.2, "Choice of
// representations"): a shift leaves the off-diagonal entries unchanged, so
// the child's LD+ is the parent's LD, stored once and copied exactly, and
// LLD+ = LD l+; otherwise LD+ = d+ l+ is formed from the child's own data.
template <class Y>
MRRR_HD double dstqds(const Y* parent, int n, Y tau, Y pivmin, Y* out, bool erep = false) {
    RepPtr<Y> P(parent, n);
    Y s = -tau;
    double growth = 0.0;
    for (int i = 0; i < n - 1; ++i) {
        Y dp = P.D[i] + s;
        if (ysmall(dp, pivmin)) dp = -pivmin;
        Y lp = qdiv<Y>(P.LD[i], dp);
        s = lp * P.L[i] * s - tau;
        double dv = to_d(dp);
        if (!isfinite(dv) || !isfinite(to_d(s))) return INFINITY;
        growth = fmax(growth, fabs(dv));
        if (out) {
            out[i] = dp;
            out[n + i] = lp;
            const Y ldp = erep ? P.LD[i] : dp * lp;
            out[2 * n + i] = ldp;
            out[3 * n + i] = ldp * lp;
        }
    }
    Y dp = P.D[n - 1] + s;
    if (ysmall(dp, pivmin)) dp = -pivmin;
    double dv = to_d(dp);
    if (!isfinite(dv)) return INFINITY;
    growth = fmax(growth, fabs(dv));
    if (out) {
        out[n - 1] = dp;
        out[2 * n - 1] = from_d<Y>(0.0);
        out[3 * n - 1] = from_d<Y>(0.0);
        out[4 * n - 1] = from_d<Y>(0.0);
    }
    return growth;
}

// ------------------------------------------------------------ twisted factorization step

// Scratch for one eigenpair: two arrays of n working-precision words,
// addressed with a stride so that the 32 eigenpairs of a warp interleave.
template <class Y> struct Scratch {
    Y* a;
    Y* b;
    int stride;
    MRRR_HD Y& A(int i) const { return a[(size_t)i * stride]; }
    MRRR_HD Y& B(int i) const { return b[(size_t)i * stride]; }
};

// accumulator for ||z||^2: at least binary64, and double-double when the
// working precision is double-double
template <class Y> struct Acc { typedef Y T; };
template <> struct Acc<float> { typedef double T; };

template <class Y> struct TwistResult {
    int r;                     // twist index (0-based), argmin |gamma_k|, smallest k on ties
    int neg;                   // negative pivots of the stationary part = negcount(lambda)
    typename Acc<Y>::T nrm2;   // ||z||^2 (z_r = 1)
};

// One twisted-factorization solve at shift lam (Sec. 2, RQI steps (i)-(iii)):
// stationary transform top-down (l+ -> A, s -> B), progressive transform
// bottom-up (gamma_k, u -> B), r = argmin |gamma_k|, then N_r^T z = e_r with z
// written into A.  Returns gamma_r through *gamma.  With r_fixed >= 0 the
// twist index is given and only rows < r of the stationary and rows > r of
// the progressive transform are formed, as one walk of n-1 rows (r
// stationary rows top-down, then the progressive rows bottom-up; both have
// the form m = b / (a + x)); the inertia of the twisted factorization,
// diag(d+_0..d+_{r-1}, gamma_r, w_{r+1}..w_{n-1}), is the Sturm count at lam
// either way (Sylvester).  If imax != null it receives the index of the
// largest |z_i| (smallest index on ties), the twist index for a next step.
template <class Y>
MRRR_HD TwistResult<Y> twisted_solve(const Y* rep, int n, Y lam, Y pivmin, const Scratch<Y>& W, Y* gamma,
                                     int r_fixed = -1, int* imax = nullptr) {
    typedef typename Acc<Y>::T A_t;
    RepPtr<Y> P(rep, n);
    TwistResult<Y> res;
    int neg = 0;
    int r;
    Y gbest;
    if (r_fixed < 0) {
        // stationary, top-down
        Y s = -lam;
        for (int i = 0; i < n - 1; ++i) {
            Y dp = P.D[i] + s;
            if (ysmall(dp, pivmin)) dp = -pivmin;
            neg += yneg(dp) ? 1 : 0;
            Y lp = qdiv<Y>(P.LD[i], dp);
            W.A(i) = lp;
            W.B(i) = s;
            s = lp * P.L[i] * s - lam;
        }
        {
            Y dp = P.D[n - 1] + s;
            if (ysmall(dp, pivmin)) dp = -pivmin;
            neg += yneg(dp) ? 1 : 0;
        }
        // progressive, bottom-up
        Y p = P.D[n - 1] - lam;
        gbest = s + p + lam;
        r = n - 1;
        for (int i = n - 2; i >= 0; --i) {
            Y om = P.LLD[i] + p;
            if (ysmall(om, pivmin)) om = -pivmin;
            Y t = qdiv<Y>(P.D[i], om);
            Y um = P.L[i] * t;
            p = p * t - lam;
            Y g = W.B(i) + p + lam;
            W.B(i) = um;
            if (!(yabs(g) > yabs(gbest))) {  // <= (NaN never wins)
                gbest = g;
                r = i;
            }
        }
    } else {
        r = r_fixed;
        const Y dlast = P.D[n - 1] - lam;
        Y x = -lam, s_r = -lam;
        if (r == 0) x = dlast;
        for (int k = 0; k < n - 1; ++k) {
            const bool st = k < r;
            const int i = st ? k : n - 2 - (k - r);
            Y den = (st ? P.D[i] : P.LLD[i]) + x;
            if (ysmall(den, pivmin)) den = -pivmin;
            neg += yneg(den) ? 1 : 0;
            const Y m = qdiv<Y>(st ? P.LD[i] : P.D[i], den);
            const Y ml = m * P.L[i];
            if (st) W.A(i) = m;
            else W.B(i) = ml;
            x = x * (st ? ml : m) - lam;
            if (k + 1 == r) {  // the stationary rows are done: s_r, then the progressive start
                s_r = x;
                x = dlast;
            }
        }
        gbest = s_r + x + lam;
        neg += yneg(gbest) ? 1 : 0;
    }
    // N_r^T z = e_r
    A_t nrm2 = A_t(1.0);
    W.A(r) = from_d<Y>(1.0);
    double zbig = 1.0;
    int im = r;
    // (a zero next to a zero or a value below 2^-900 is the underflowed tail
    // of a localized vector: it stays zero, without reviving subnormals)
    const double ztiny = 0x1p-900;
    for (int i = r - 1; i >= 0; --i) {
        Y zn = W.A(i + 1);
        Y z;
        if (to_d(zn) == 0.0 && i + 2 < n) {
            // row i+1 of the tridiagonal with z_{i+1} = 0: e_i z_i + e_{i+1} z_{i+2} = 0
            z = fabs(to_d(W.A(i + 2))) < ztiny ? from_d<Y>(0.0) : -(P.LD[i + 1] / P.LD[i]) * W.A(i + 2);
        } else {
            z = -(W.A(i) * zn);
        }
        W.A(i) = z;
        A_t za = A_t(z);
        nrm2 += za * za;
        double az = fabs(to_d(z));
        if (az >= zbig) {  // walking down: >= keeps the smallest index on ties
            zbig = az;
            im = i;
        }
    }
    for (int i = r; i < n - 1; ++i) {
        Y zc = W.A(i);
        Y z;
        if (to_d(zc) == 0.0 && i >= 1) {
            // row i with z_i = 0: e_{i-1} z_{i-1} + e_i z_{i+1} = 0
            z = fabs(to_d(W.A(i - 1))) < ztiny ? from_d<Y>(0.0) : -(P.LD[i - 1] / P.LD[i]) * W.A(i - 1);
        } else {
            z = -(W.B(i) * zc);
        }
        W.A(i + 1) = z;
        A_t za = A_t(z);
        nrm2 += za * za;
        double az = fabs(to_d(z));
        if (az > zbig) {
            zbig = az;
            im = i + 1;
        }
    }
    if (imax) *imax = im;
    res.r = r;
    res.neg = neg;
    res.nrm2 = nrm2;
    *gamma = gbest;
    return res;
}

}  // namespace mrrr
