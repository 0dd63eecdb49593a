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
//  * The count carries the stationary transform in projective form (a
//    numerator and a denominator) and needs no divide; in the twisted
//    factorization the divide is a reciprocal estimate with Newton-Raphson
//    refinement fused into the next operation (see qdiv).
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

// Guarded fallback, kept out of line so that it does not weigh on the
// register allocation and scheduling of the unguarded hot loops.
static __device__ __noinline__ int negcount_guarded(const double* D, const double* LLD, int n, double tau, double pivmin) {
    return negcount<double>(D, LLD, n, tau, pivmin);
}

// 1 if x is zero, subnormal, infinite or NaN (from the high word)
__device__ __forceinline__ unsigned dnotnormal(double x) {
    return (((unsigned)__double2hiint(x) & 0x7ff00000u) - 0x00100000u) >= 0x7fe00000u ? 1u : 0u;
}

// Power-of-two scaling of the projective recurrences: k with |x| 2^k in
// [1, 2) for a normal x, clamped so that 2^k is normal (x is not normal only
// on a path whose result is discarded), and 2^k for k in [-1022, 1023].
__device__ __forceinline__ int dscale_exp(double x) {
    const int e = (int)(((unsigned)__double2hiint(x) >> 20) & 0x7ffu);
    return max(1023 - e, -1022);
}
__device__ __forceinline__ double dpow2(int k) { return __hiloint2double((k + 1023) << 20, 0); }

// A projective pair is rescaled when |X| leaves [2^-256, 2^256): a row
// changes |X| by the pivot d+_i, so X stays normal unless a single pivot is
// below ~2^-760.  A zero or subnormal X (a vanished pivot) is left as it is:
// the projective recurrences need no special case for it.
__device__ __forceinline__ bool dneeds_rescale(double x) {
    const unsigned e = ((unsigned)__double2hiint(x) >> 20) & 0x7ffu;
    return e != 0u && e - (1023u - 256u) >= 512u;
}

// x 2^k by integer arithmetic on the exponent field, so that a rescale
// costs no FP64 issue slot.  On this GPU an FP64 multiply under a false
// predicate holds the FP64 pipe as long as an executed one, and the
// per-row rescale tests of the twisted walk and solve are if-converted: a
// multiply there would cost every row a slot.  Exact wherever x 2^k is a
// normal number; a zero or subnormal x, or a result below the normal range,
// becomes a zero of the same sign (the projective values it scales are then
// negligible next to the ones kept), a result above it becomes an infinity
// (which the callers' final finiteness checks catch), and an infinity or
// NaN stays as it is.
// x = m 2^e with |m| in [1, 2): returns m (x's exponent field set to that of
// 1) and e, for a normal x, by integer arithmetic.
__device__ __forceinline__ double dsplit_exp(double x, int& e) {
    const unsigned hi = (unsigned)__double2hiint(x);
    e = (int)((hi >> 20) & 0x7ffu) - 1023;
    return __hiloint2double((int)((hi & 0x800fffffu) | 0x3ff00000u), __double2loint(x));
}

__device__ __forceinline__ double dscale_bits(double x, int k) {
    const unsigned hi = (unsigned)__double2hiint(x);
    const int e = (int)((hi >> 20) & 0x7ffu);
    const int en = e + k;
    const unsigned sgn = hi & 0x80000000u;
    const bool keep = e == 0x7ff;
    const bool zero = !keep && (e == 0 || en <= 0);
    const bool inf = !keep && !zero && en >= 0x7ff;
    const unsigned nhi = keep ? hi : zero ? sgn : inf ? (sgn | 0x7ff00000u) : hi + ((unsigned)k << 20);
    const int nlo = (keep || !(zero || inf)) ? __double2loint(x) : 0;
    return __hiloint2double((int)nhi, nlo);
}
// Sturm count (number of eigenvalues of L D L^T below tau) for bisection and
// bracket checks, without a divide.  The stationary transform maps s_i to
// s_{i+1} = lld_i s_i / (d_i + s_i) - tau, a linear fractional map; writing
// s_i = N_i / P_{i-1} (P_{-1} = 1, N_0 = -tau) turns it into the linear
// recurrence
//     P_i     = d_i P_{i-1} + N_i          (so d+_i = d_i + s_i = P_i / P_{i-1})
//     N_{i+1} = lld_i N_i - tau P_i
// and d+_i < 0 exactly when P_i and P_{i-1} have opposite signs.  With fused
// multiply-adds d+_i is rounded once (as in the divide form) and s_{i+1}
// twice (three times in the divide form), so the count is exact for the rep
// perturbed element-wise by a few ulps -- the mixed relative stability of the
// stationary qd transform (Sec. 2).  A row costs three FP64 instructions, two
// of them on the dependency chain, against five and a reciprocal estimate for
// the divide form.  Only the ratio N/P and the sign of P matter, so every
// sixteen rows both are scaled by the power of two that brings P into [1, 2)
// (after preprocessing a row changes |P| by a pivot of modest size).  A
// vanished pivot needs no special case: P_i = +-0 counts d+_i as a pivot of
// that sign and the recurrence continues from N_{i+1} = lld_i N_i (the limit
// of the divide form).  An overflow, or an underflow that leaves P zero or
// subnormal at a rescaling point (where the pair could have vanished
// altogether and lost the count), sends the count to the guarded divide
// form.
__device__ __forceinline__ int negcount_fast(const double* __restrict__ D, const double* __restrict__ LLD, int n,
                                             double tau, double pivmin) {
    const double mtau = -tau;
    double P = 1.0, N = mtau;
    unsigned hp = 0u;  // high word of P_{i-1}
    int cnt = 0;
    unsigned bad = 0u;
    int i = 0;
    for (; i + 8 <= n - 1; i += 8) {
        const int ip = min(i + kPrefetch, n - 1);
        pf_l2(D + ip);
        pf_l2(LLD + ip);
        double d[8], l[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            d[k] = __ldg(D + i + k);
            l[k] = __ldg(LLD + i + k);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const double a = l[k] * N;
            P = fma(d[k], P, N);
            const unsigned h = (unsigned)__double2hiint(P);
            cnt += (int)((h ^ hp) >> 31);
            hp = h;
            N = fma(mtau, P, a);
        }
        if (i & 8) {  // every sixteen rows (the same rows in every lane)
            bad |= dnotnormal(P);
            const double f = dpow2(dscale_exp(P));
            P *= f;
            N *= f;
        }
    }
    for (; i < n - 1; ++i) {
        const double a = __ldg(LLD + i) * N;
        P = fma(__ldg(D + i), P, N);
        const unsigned h = (unsigned)__double2hiint(P);
        cnt += (int)((h ^ hp) >> 31);
        hp = h;
        N = fma(mtau, P, a);
    }
    P = fma(__ldg(D + n - 1), P, N);
    cnt += (int)((((unsigned)__double2hiint(P)) ^ hp) >> 31);
    if (bad | dnotnormal(P) | !dfinite(N)) return negcount_guarded(D, LLD, n, tau, pivmin);
    return cnt;
}

// Guarded double-double count (out of line) for the projective one's
// fallback.
static __device__ __noinline__ int negcount_dd_guarded(const dd* D, const dd* LLD, int n, dd tau, dd pivmin) {
    return negcount<dd>(D, LLD, n, tau, pivmin);
}

// The double-double Sturm count in the projective form of negcount_fast:
//     P_i = d_i P_{i-1} + N_i,   N_{i+1} = lld_i N_i - tau P_i,
// a pivot negative where P changes sign.  Each row is three double-double
// products and two sums (about 60 binary64 instructions) instead of a sum, a
// product and a double-double division (about 140): the division alone is
// three binary64 divisions and three double-double sums.  Every operation is
// rounded once in double-double, so the count is exact for the
// representation perturbed element-wise by a few units of 2^-104 -- the mixed
// relative stability of Sec. 2.  The pair is rescaled every sixteen rows by
// the power of two that brings the high word of P into [1, 2); an overflow,
// or a P that is zero or subnormal at a rescaling point or at the end, sends
// the count to the guarded divide form.
__device__ __forceinline__ int negcount_dd_fast(const dd* __restrict__ D, const dd* __restrict__ LLD, int n, dd tau,
                                                dd pivmin) {
    const dd mtau = -tau;
    dd P(1.0), N = mtau;
    unsigned hp = 0u;  // high word of P_{i-1}.hi
    int cnt = 0;
    unsigned bad = 0u;
    auto row = [&](int i) {
        const dd a = LLD[i] * N;
        P = D[i] * P + N;
        const unsigned h = (unsigned)__double2hiint(P.hi);
        cnt += (int)((h ^ hp) >> 31);
        hp = h;
        N = a + mtau * P;
    };
    int i = 0;
    for (; i + 16 <= n - 1; i += 16) {  // sixteen rows, then the rescale
        const int ip = min(i + kPrefetch, n - 1);
        pf_l2(D + ip);
        pf_l2(LLD + ip);
#pragma unroll 4
        for (int k = 0; k < 16; ++k) row(i + k);
        bad |= dnotnormal(P.hi);
        const double f = dpow2(dscale_exp(P.hi));
        P = dd(P.hi * f, P.lo * f);
        N = dd(N.hi * f, N.lo * f);
    }
    for (; i < n - 1; ++i) row(i);
    P = D[n - 1] * P + N;
    cnt += (int)((((unsigned)__double2hiint(P.hi)) ^ hp) >> 31);
    if (bad | dnotnormal(P.hi) | !dfinite(N.hi)) return negcount_dd_guarded(D, LLD, n, tau, pivmin);
    return cnt;
}

// The low-precision Sturm count of the pre-bisection (binary32 under a
// binary64 working precision, see negcount_lo) in the same projective form
// as negcount_fast: two dependent FMAs per row instead of an add, a divide
// and a subtract.  binary32 has a narrower exponent range, so the pair is
// rescaled every four rows; an overflow, or a P that is zero or subnormal at
// a rescaling point or at the end, falls back to the divide form.  Its
// brackets are verified in the working precision.
static __device__ __noinline__ int negcount_lo_guarded(const float* D, const float* LLD, int n, float tau,
                                                       float pivmin) {
    return negcount_lo<float>(D, LLD, n, tau, pivmin);
}

__device__ __forceinline__ int negcount_lo_fast(const float* __restrict__ D, const float* __restrict__ LLD, int n,
                                                float tau, float pivmin) {
    const float mtau = -tau;
    float P = 1.0f, N = mtau;
    unsigned hp = 0u;  // bits of P_{i-1}
    int cnt = 0;
    unsigned bad = 0u;
    int i = 0;
    for (; i + 8 <= n - 1; i += 8) {
        const int ip = min(i + kPrefetch, n - 1);
        pf_l2(D + ip);
        pf_l2(LLD + ip);
        float d[8], l[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            d[k] = __ldg(D + i + k);
            l[k] = __ldg(LLD + i + k);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float a = l[k] * N;
            P = fmaf(d[k], P, N);
            const unsigned h = __float_as_uint(P);
            cnt += (int)((h ^ hp) >> 31);
            hp = h;
            N = fmaf(mtau, P, a);
            if ((k & 3) == 3) {
                // every four rows: scale by 2^q with |P| 2^q in [1, 2), q
                // clamped so that 2^q is normal
                const int e = (int)((hp >> 23) & 0xffu);
                bad |= (unsigned)(e == 0 || e == 255);
                const int q = max(127 - e, -126);
                const float f = __uint_as_float((unsigned)(q + 127) << 23);
                P *= f;
                N *= f;
            }
        }
    }
    for (; i < n - 1; ++i) {
        const float a = __ldg(LLD + i) * N;
        P = fmaf(__ldg(D + i), P, N);
        const unsigned h = __float_as_uint(P);
        cnt += (int)((h ^ hp) >> 31);
        hp = h;
        N = fmaf(mtau, P, a);
    }
    P = fmaf(__ldg(D + n - 1), P, N);
    cnt += (int)((__float_as_uint(P) ^ hp) >> 31);
    const unsigned ee = (__float_as_uint(P) >> 23) & 0xffu;
    if (bad | (unsigned)(ee == 0u || ee == 255u) | (unsigned)!isfinite(N))
        return negcount_lo_guarded(D, LLD, n, tau, pivmin);
    return cnt;
}

// First twist index of an RQI step from the binary32 copy of the rep
// (Sec. 2, "Rayleigh quotient iteration": r = argmin_k |gamma_k| with
// gamma_k = s_k + p_k + tau, from the stationary and the progressive
// transform at tau), in projective form: s_i = N_i / P_{i-1} as in
// negcount_lo_fast, and p_i = Q_i / R_{i+1} with R_n = 1,
// Q_{n-1} = d_{n-1} - tau,
//     R_{i+1} = lld_i R_{i+2} + Q_{i+1}     (= R_{i+2} (lld_i + p_{i+1}))
//     Q_i     = d_i Q_{i+1} - tau R_{i+1}   (so p_i = d_i p_{i+1} / (lld_i + p_{i+1}) - tau).
// A row's dependency chain is two FMAs; the ratios come from approximate
// reciprocals off the chain (only the position of the smallest |gamma_k|
// matters).  Both pairs are rescaled by a power of two every four rows.
// s_k is kept in s_store for the bottom-up pass.  Returns r (smallest index
// on ties), or -1 when a rescaling point met a zero, subnormal or
// non-finite value, or no gamma_k is finite (the caller then factors in the
// working precision).
__device__ __forceinline__ int twist_index_lo_fast(const float* __restrict__ D, const float* __restrict__ LLD,
                                                   int n, float tau, float* __restrict__ s_store) {
    const float mtau = -tau;
    unsigned bad = 0u;
    auto rescale = [&](float& u, float& v) {
        const int e = (int)((__float_as_uint(u) >> 23) & 0xffu);
        bad |= (unsigned)(e == 0 || e == 255);
        const float f = __uint_as_float((unsigned)(max(127 - e, -126) + 127) << 23);
        u *= f;
        v *= f;
    };
    // stationary, top-down
    float P = 1.0f, N = mtau;
    int i = 0;
    for (; i + 8 <= n - 1; i += 8) {
        const int ip = min(i + kPrefetch, n - 1);
        pf_l2(D + ip);
        pf_l2(LLD + ip);
        float d[8], l[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            d[k] = __ldg(D + i + k);
            l[k] = __ldg(LLD + i + k);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            s_store[i + k] = __fdividef(N, P);
            const float a = l[k] * N;
            P = fmaf(d[k], P, N);
            N = fmaf(mtau, P, a);
            if ((k & 3) == 3) rescale(P, N);
        }
    }
    for (; i < n - 1; ++i) {
        s_store[i] = __fdividef(N, P);
        const float a = __ldg(LLD + i) * N;
        P = fmaf(__ldg(D + i), P, N);
        N = fmaf(mtau, P, a);
    }
    rescale(P, N);
    const float s_last = __fdividef(N, P);
    // progressive, bottom-up, with the running arg-min of |gamma_k|
    float R = 1.0f, Q = __ldg(D + n - 1) - tau;
    float gbest = s_last + Q + tau;
    int r = n - 1;
    auto row = [&](int j, float dj, float lj, float sj) {
        const float t = dj * Q;
        R = fmaf(lj, R, Q);
        Q = fmaf(mtau, R, t);
        const float g = sj + __fdividef(Q, R) + tau;
        if (fabsf(g) <= fabsf(gbest)) {  // smallest index on ties (the walk goes down)
            gbest = g;
            r = j;
        }
    };
    i = n - 2;
    for (; i - 7 >= 0; i -= 8) {
        const int ip = max(i - kPrefetch, 0);
        pf_l2(D + ip);
        pf_l2(LLD + ip);
        pf_l2(s_store + ip);
        float d[8], l[8], sv[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            d[k] = __ldg(D + i - k);
            l[k] = __ldg(LLD + i - k);
            sv[k] = s_store[i - k];
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            row(i - k, d[k], l[k], sv[k]);
            if ((k & 3) == 3) rescale(R, Q);
        }
    }
    for (; i >= 0; --i) row(i, __ldg(D + i), __ldg(LLD + i), s_store[i]);
    rescale(R, Q);
    if (bad || !isfinite(gbest)) return -1;
    return r;
}

// Pre-bisection count for the low precision Lo of the device path
template <class Lo>
__device__ __forceinline__ int count_lo(const Lo* D, const Lo* LLD, int n, Lo tau, Lo pivmin) {
    if constexpr (std::is_same<Lo, float>::value) return negcount_lo_fast(D, LLD, n, tau, pivmin);
    else if constexpr (std::is_same<Lo, double>::value) return negcount_fast(D, LLD, n, tau, pivmin);
    else return negcount_lo<Lo>(D, LLD, n, tau, pivmin);
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
                                             float* out_lo, bool erep) {
    double g = dstqds<double>(parent, n, tau, pivmin, out, erep);
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
                                              double* __restrict__ out, float* __restrict__ out_lo, bool erep = false) {
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
            const double ldp = erep ? ldi : dp * lp;  // e-representation: the parent's LD, exactly
            const double lldp = ldp * lp;
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
        return dstqds_guarded(parent, n, tau, pivmin, out, out_lo, erep);
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

// steps of the twisted walk and solve whose operands are loaded ahead
constexpr int kGp = 4;

// Twisted factorization at a given twist index r in projective form, and
// the solve N_r^T z = e_r (Sec. 2, RQI steps (i)-(iii)), without a divide
// per row.
//
// The stationary rows i < r carry s_i = N_i / P_{i-1} (P_{-1} = 1,
// N_0 = -lam):  P_i = d_i P_{i-1} + N_i (so d+_i = P_i / P_{i-1}) and
// N_{i+1} = lld_i N_i - lam P_i, as in negcount_fast.  The progressive rows
// i = n-2 .. r carry p_{i+1} = Q_{i+1} / R_{i+2} (R_n = 1,
// Q_{n-1} = d_{n-1} - lam):  R_{i+1} = lld_i R_{i+2} + Q_{i+1} (so the pivot
// of the progressive factorization is R_{i+1} / R_{i+2}) and
// Q_i = d_i Q_{i+1} - lam R_{i+1}.  Both are one walk of n-1 steps per lane
// -- r stationary rows top-down, then the progressive rows bottom-up -- of
// the same form X' = a X + Y, Y' = b Y - lam X' with (a, b) = (d_i, lld_i)
// or (lld_i, d_i), so that lanes with different r do not diverge.  A pivot
// is negative where X changes sign; gamma_r = s_r + p_r + lam takes the
// only two divides.
//
// With l+_i = ld_i P_{i-1} / P_i and u_i = ld_i R_{i+2} / R_{i+1} the solve
// telescopes: z_i = w_i P_{i-1} for i < r with w_r = 1 / P_{r-1},
// w_i = -ld_i w_{i+1}, and z_i = v_i R_{i+1} for i > r with
// v_r = 1 / R_{r+1}, v_{i+1} = -ld_i v_i.  The walk stores the multiplier of
// z_i (P_{i-1} or R_{i+1}) in A[i]; the solve overwrites it with z_i.  A
// vanished pivot needs no special rule here (z_{i+1} = 0 and z_i follow
// from the neighbouring multipliers), and entries of z below the normal
// range (the tail of a localized vector) are zero.
//
// Where X leaves [2^-256, 2^256), X and Y are scaled by the power of two 2^k
// that brings X into [1, 2) -- the ratios and the signs do not change --
// right after X was stored, so that both the decision and k follow from the
// stored value itself; the walk scales on the exponent fields (dscale_bits).
// The solve keeps its running factor as a mantissa in [1, 2) and an integer
// exponent, and reaching that entry adds k to the exponent.  Neither costs
// an FP64 instruction, and the factor cannot underflow between two
// far-apart peaks of the vector.  An overflow, or a vanished pivot at the
// twist (P_{r-1} or R_{r+1} zero), sends the step to the guarded generic
// solve.
__device__ __forceinline__ TwistResult<double> twisted_fixed_proj(const double* __restrict__ rep, int n, double lam,
                                                                 double pivmin, double* __restrict__ A,
                                                                 double* __restrict__ B, double* gamma, int* imax,
                                                                 int r) {
    const double* __restrict__ D = rep;
    const double* __restrict__ LD = rep + 2 * n;
    const double* __restrict__ LLD = rep + 3 * n;
    const double mlam = -lam;
    const int steps = n - 1;
    int neg = 0;
    // walk step k: row k of the stationary chain for k < r, else row
    // n-2-(k-r) of the progressive one
    auto wrow = [&](int k) { return k < r ? k : n - 2 - (k - r); };
    // top chain state (P_{i-1}, N_i); for r = 0 the chain is empty
    double X = 1.0, Y = r > 0 ? mlam : __ldg(D + n - 1) - lam;
    double Xtop = 1.0, Ytop = mlam;
    unsigned hx = (unsigned)__double2hiint(X);
    // steps in whole groups of kGp (their operands loaded a group ahead,
    // with no per-step bounds test), then the remaining steps
    const int full = steps - steps % kGp;
    auto wstep = [&](int k, double a, double b) {
        const bool st = k < r;
        const int i = wrow(k);
        A[st ? i : i + 1] = X;
        if (dneeds_rescale(X)) {
            const int q = dscale_exp(X);
            X = dscale_bits(X, q);
            Y = dscale_bits(Y, q);
        }
        const double t = b * Y;
        X = fma(a, X, Y);
        const unsigned h = (unsigned)__double2hiint(X);
        neg += (int)((h ^ hx) >> 31);
        hx = h;
        Y = fma(mlam, X, t);
        if (k + 1 == r) {  // the stationary rows are done: the progressive chain starts
            Xtop = X;
            Ytop = Y;
            X = 1.0;
            Y = __ldg(D + n - 1) - lam;
            hx = (unsigned)__double2hiint(X);
        }
    };
    // operands of walk step k (clamped to a valid row past the end)
    auto wload = [&](int k, double& a, double& b) {
        const int kc = min(k, steps - 1);
        const int i = wrow(kc);
        const bool st = kc < r;
        a = __ldg((st ? D : LLD) + i);
        b = __ldg((st ? LLD : D) + i);
    };
    double ca[kGp], cb[kGp], na[kGp], nb[kGp];
    if (full > 0) {
#pragma unroll
        for (int q = 0; q < kGp; ++q) wload(q, ca[q], cb[q]);
    }
    for (int k0 = 0; k0 < full; k0 += kGp) {
        {
            const int ipf = wrow(min(k0 + kPrefetch, steps - 1));
            pf_l2(D + ipf);
            pf_l2(LLD + ipf);
        }
#pragma unroll
        for (int q = 0; q < kGp; ++q) wload(k0 + kGp + q, na[q], nb[q]);
#pragma unroll
        for (int q = 0; q < kGp; ++q) wstep(k0 + q, ca[q], cb[q]);
#pragma unroll
        for (int q = 0; q < kGp; ++q) {
            ca[q] = na[q];
            cb[q] = nb[q];
        }
    }
    for (int k = full; k < steps; ++k) {
        double a, b;
        wload(k, a, b);
        wstep(k, a, b);
    }
    // the progressive chain ends at R_{r+1} (R_n = 1 for r = n-1)
    const double gam = Ytop / Xtop + Y / X + lam;
    neg += dsign(gam);
    // an overflow leaves the chain non-finite; a vanished pivot at the twist
    // leaves no finite gamma_r
    if (dnotnormal(Xtop) | dnotnormal(X) | !dfinite(gam)) return twisted_guarded(rep, n, lam, pivmin, A, B, gamma, imax);
    // solve: step k computes z_iz, iz = r-1-k downward (k < r), then
    // iz = k+1 upward; the coefficient is ld_iz downward, ld_{iz-1} upward.
    // The arg-max of |z| (smallest index on ties) is exact: it is the next
    // twist index and also fixes the sign of the stored vector (largest entry
    // positive).
    auto sz = [&](int k) { return k < r ? r - 1 - k : k + 1; };
    auto sl = [&](int k) { return k < r ? r - 1 - k : k; };
    A[r] = 1.0;
    double nrm2 = 1.0;
    unsigned long long zmax = dabsbits(1.0);
    int im = r;
    // the running factor is f 2^fe with |f| in [1, 2): it can fall below the
    // normal range between two far-apart peaks of the vector and rise again,
    // so it is kept as a mantissa and an integer exponent, which also makes
    // the walk's rescalings (2^q at the rows where the stored multiplier
    // left the window) integer additions; only z itself is rounded into
    // binary64 (an entry below the normal range becomes zero)
    int fe, vre;
    double f = dsplit_exp(1.0 / Xtop, fe);  // w_r
    const double vr = dsplit_exp(1.0 / X, vre);
    auto sstep = [&](int k, double a, double l) {
        const int iz = sz(k);
        if (k == r) {  // the upward walk restarts at v_r
            f = vr;
            fe = vre;
        }
        int e;
        f = dsplit_exp(-(l * f), e);
        fe += e + (dneeds_rescale(a) ? dscale_exp(a) : 0);
        const double z = dscale_bits(f * a, fe);
        A[iz] = z;
        nrm2 = fma(z, z, nrm2);
        const unsigned long long za = dabsbits(z);
        const bool better = za > zmax || (za == zmax && iz < im);
        zmax = better ? za : zmax;
        im = better ? iz : im;
    };
    auto sload = [&](int k, double& a, double& l) {
        const int kc = min(k, steps - 1);
        a = A[sz(kc)];
        l = __ldg(LD + sl(kc));
    };
    if (full > 0) {
#pragma unroll
        for (int q = 0; q < kGp; ++q) sload(q, ca[q], cb[q]);
    }
    for (int k0 = 0; k0 < full; k0 += kGp) {
        {
            const int kp = min(k0 + kPrefetch, steps - 1);
            pf_l2(A + sz(kp));
            pf_l2(LD + sl(kp));
        }
#pragma unroll
        for (int q = 0; q < kGp; ++q) sload(k0 + kGp + q, na[q], nb[q]);
#pragma unroll
        for (int q = 0; q < kGp; ++q) sstep(k0 + q, ca[q], cb[q]);
#pragma unroll
        for (int q = 0; q < kGp; ++q) {
            ca[q] = na[q];
            cb[q] = nb[q];
        }
    }
    for (int k = full; k < steps; ++k) {
        double a, l;
        sload(k, a, l);
        sstep(k, a, l);
    }
    *imax = im;
    TwistResult<double> res;
    res.r = r;
    res.neg = neg;
    res.nrm2 = nrm2;
    *gamma = gam;
    return res;
}

// Guarded generic double-double twisted solve (out of line) at a given twist
// index, with the arg-max of |z| (the projective step's fallback).
static __device__ __noinline__ TwistResult<dd> twisted_dd_guarded(const dd* rep, int n, dd lam, dd pivmin,
                                                                 const Scratch<dd>& W, dd* gamma, int r, int* imax) {
    return twisted_solve<dd>(rep, n, lam, pivmin, W, gamma, r, imax);
}

// The fixed-r twisted step of twisted_fixed_proj in double-double: the same
// projective walk (X' = a X + Y, Y' = b Y - lam X', r stationary rows
// top-down, then the progressive rows bottom-up) and the same telescoped
// solve (z_i = w_i P_{i-1}, w_i = -ld_i w_{i+1}; below r with R_{i+1}), with
// no division per row: a row of the walk is three double-double products
// and two sums (about 60 binary64 instructions) against a double-double
// division, a sum and two products (about 150) in the generic step.  gamma_r
// = N_r / P_{r-1} + Q_r / R_{r+1} + lam takes the step's only two divisions.
// X is rescaled by a power of two where it leaves [2^-256, 2^256), right
// after it was stored, and the solve multiplies its running factor by the
// same power where it meets that stored value.  An overflow, or a vanished
// pivot at the twist, sends the step to the generic solve.
__device__ __forceinline__ TwistResult<dd> twisted_fixed_proj_dd(const dd* __restrict__ rep, int n, dd lam,
                                                                dd pivmin, const Scratch<dd>& W, dd* gamma,
                                                                int* imax, int r) {
    const dd* __restrict__ D = rep;
    const dd* __restrict__ LD = rep + 2 * n;
    const dd* __restrict__ LLD = rep + 3 * n;
    dd* __restrict__ A = W.a;
    const dd mlam = -lam;
    const int steps = n - 1;
    int neg = 0;
    auto wrow = [&](int k) { return k < r ? k : n - 2 - (k - r); };
    const dd ylast = D[n - 1] - lam;
    dd X(1.0), Y = r > 0 ? mlam : ylast;
    dd Xtop(1.0), Ytop = mlam;
    unsigned hx = (unsigned)__double2hiint(X.hi);
    for (int k = 0; k < steps; ++k) {
        if ((k & 15) == 0) {
            const int ip = wrow(min(k + kPrefetch, steps - 1));
            pf_l2(D + ip);
            pf_l2(LLD + ip);
        }
        const bool st = k < r;
        const int i = wrow(k);
        const dd a = st ? D[i] : LLD[i];
        const dd b = st ? LLD[i] : D[i];
        A[st ? i : i + 1] = X;
        if (dneeds_rescale(X.hi)) {
            const int q = dscale_exp(X.hi);
            X = dd(dscale_bits(X.hi, q), dscale_bits(X.lo, q));
            Y = dd(dscale_bits(Y.hi, q), dscale_bits(Y.lo, q));
        }
        const dd t = b * Y;
        X = a * X + Y;
        const unsigned h = (unsigned)__double2hiint(X.hi);
        neg += (int)((h ^ hx) >> 31);
        hx = h;
        Y = t + mlam * X;
        if (k + 1 == r) {  // the stationary rows are done: the progressive chain starts
            Xtop = X;
            Ytop = Y;
            X = dd(1.0);
            Y = ylast;
            hx = (unsigned)__double2hiint(X.hi);
        }
    }
    const dd gam = Ytop / Xtop + Y / X + lam;
    neg += dsign(gam.hi);
    if (dnotnormal(Xtop.hi) | dnotnormal(X.hi) | !dfinite(gam.hi))
        return twisted_dd_guarded(rep, n, lam, pivmin, W, gamma, r, imax);
    // solve: z_r = 1, then from r outwards (down, then up)
    A[r] = dd(1.0);
    dd nrm2(1.0);
    unsigned long long zmax = dabsbits(1.0);
    int im = r;
    // the running factor is f 2^fe with |f.hi| in [1, 2), as in the binary64
    // step: it neither underflows between far-apart peaks nor needs an FP64
    // instruction to rescale
    auto split = [](dd& f, int& fe) {
        int e;
        const double h = dsplit_exp(f.hi, e);
        f = dd(h, dscale_bits(f.lo, -e));
        fe = e;
    };
    int fe = 0;
    auto sstep = [&](dd& f, int iz, int il) {
        const dd av = A[iz];
        f = -(LD[il] * f);
        int e;
        split(f, e);
        fe += e + (dneeds_rescale(av.hi) ? dscale_exp(av.hi) : 0);
        const dd zm = f * av;
        const dd z = dd(dscale_bits(zm.hi, fe), dscale_bits(zm.lo, fe));
        A[iz] = z;
        nrm2 = nrm2 + z * z;
        const unsigned long long za = dabsbits(z.hi);
        const bool better = za > zmax;
        zmax = better ? za : zmax;
        im = better ? iz : im;
    };
    dd f = dd(1.0) / Xtop;  // w_r
    split(f, fe);
    for (int iz = r - 1; iz >= 0; --iz) {
        if (((r - 1 - iz) & 15) == 0) pf_l2(A + max(iz - kPrefetch, 0));
        sstep(f, iz, iz);
    }
    f = dd(1.0) / X;  // v_r
    split(f, fe);
    for (int iz = r + 1; iz < n; ++iz) {
        if (((iz - r - 1) & 15) == 0) pf_l2(A + min(iz + kPrefetch, n - 1));
        sstep(f, iz, iz - 1);
    }
    *imax = im;
    *gamma = gam;
    TwistResult<dd> res;
    res.r = r;
    res.neg = neg;
    res.nrm2 = nrm2;
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
// progressive transform are needed -- one pass instead of two, in the
// projective form of twisted_fixed_proj.  In both
// cases the inertia of Delta_r = diag(d+_0..d+_{r-1}, gamma_r,
// w_{r+1}..w_{n-1}) is the Sturm count at lam (Sylvester), used to update
// the bisection bracket.
__device__ __forceinline__ TwistResult<double> twisted_solve_fast(const double* __restrict__ rep, int n, double lam,
                                                                 double pivmin, double* __restrict__ A,
                                                                 double* __restrict__ B, double* gamma, int* imax,
                                                                 int r_fixed = -1) {
    if (r_fixed >= 0) return twisted_fixed_proj(rep, n, lam, pivmin, A, B, gamma, imax, r_fixed);
    const double* __restrict__ D = rep;
    const double* __restrict__ L = rep + n;
    const double* __restrict__ LD = rep + 2 * n;
    const double* __restrict__ LLD = rep + 3 * n;
    TwistResult<double> res;
    int neg = 0;
    int r;
    double gbest;
    bool bad;
    {
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
