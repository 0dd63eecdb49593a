// Double-double arithmetic (a value is the unevaluated sum hi + lo of two
// binary64 numbers, |lo| <= ulp(hi)/2, about 106 significant bits).
//
// This is the working precision y of the solver for binary64 input/output:
// it takes the place of the software binary128 the paper uses for its
// "double/quadruple" solver (Sec. 4.1), with unit roundoff ~2^-104 instead of
// 2^-113, which still satisfies n eps_y <= eps_x sqrt(n) (Sec. 3.2, footnote
// on the simplification of Theorem 1) for every n this library accepts.
//
// The building blocks are the error-free transformations
//   two_sum      (Knuth, TAOCP vol. 2, Sec. 4.2.2): a + b = s + err exactly,
//   fast_two_sum (Dekker 1971, needs |a| >= |b|),
//   two_prod     (a*b = p + err exactly, with err from one fused multiply-add),
// and the double-double operations are the "accurate" variants described by
// Hida, Li and Bailey, "Algorithms for quad-double precision floating point
// arithmetic" (ARITH-15, 2001): addition renormalises twice so that the
// relative error stays O(2^-104) even under cancellation, which the
// element-wise mixed relative stability of the qd transforms (Sec. 2,
// "Shifting the spectrum") relies on; division is long division with two
// correction quotients.
#pragma once

#include <cfloat>
#include <algorithm>
#include <cmath>

#if defined(__CUDACC__)
#define MRRR_HD __host__ __device__ __forceinline__
#else
#define MRRR_HD inline
#endif

namespace mrrr {

#if !defined(__CUDACC__)
using std::fabs;
using std::fma;
using std::fmax;
using std::fmin;
using std::frexp;
using std::isfinite;
using std::ldexp;
using std::max;
using std::min;
using std::nextafter;
using std::sqrt;
#endif

struct dd {
    double hi, lo;
    dd() = default;
    MRRR_HD constexpr dd(double h) : hi(h), lo(0.0) {}
    MRRR_HD constexpr dd(double h, double l) : hi(h), lo(l) {}
};

MRRR_HD dd two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double err = (a - (s - bb)) + (b - bb);
    return dd(s, err);
}

MRRR_HD dd fast_two_sum(double a, double b) {
    double s = a + b;
    double err = b - (s - a);
    return dd(s, err);
}

MRRR_HD dd two_prod(double a, double b) {
    double p = a * b;
    double err = fma(a, b, -p);
    return dd(p, err);
}

MRRR_HD dd operator+(const dd& x, const dd& y) {
    dd s = two_sum(x.hi, y.hi);
    dd t = two_sum(x.lo, y.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}

MRRR_HD dd operator-(const dd& x) { return dd(-x.hi, -x.lo); }
MRRR_HD dd operator-(const dd& x, const dd& y) { return x + (-y); }

MRRR_HD dd operator*(const dd& x, const dd& y) {
    dd p = two_prod(x.hi, y.hi);
    p.lo = fma(x.hi, y.lo, p.lo);
    p.lo = fma(x.lo, y.hi, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

// dd times a double (one product fewer)
MRRR_HD dd mul_d(const dd& x, double y) {
    dd p = two_prod(x.hi, y);
    p.lo = fma(x.lo, y, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

MRRR_HD dd operator/(const dd& x, const dd& y) {
    // long division: q1 = x/y in double, r = x - q1*y exactly enough, etc.
    double q1 = x.hi / y.hi;
    dd r = x - mul_d(y, q1);
    double q2 = r.hi / y.hi;
    r = r - mul_d(y, q2);
    double q3 = r.hi / y.hi;
    dd q = fast_two_sum(q1, q2);
    return q + dd(q3);
}

MRRR_HD dd& operator+=(dd& x, const dd& y) { x = x + y; return x; }
MRRR_HD dd& operator-=(dd& x, const dd& y) { x = x - y; return x; }
MRRR_HD dd& operator*=(dd& x, const dd& y) { x = x * y; return x; }

// Ordering by value.  For a normalised dd, sign(x) = sign(hi) unless hi = 0.
MRRR_HD bool operator<(const dd& x, const dd& y) { return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo); }
MRRR_HD bool operator>(const dd& x, const dd& y) { return y < x; }
MRRR_HD bool operator<=(const dd& x, const dd& y) { return !(y < x); }
MRRR_HD bool operator>=(const dd& x, const dd& y) { return !(x < y); }

MRRR_HD dd dd_abs(const dd& x) { return x.hi < 0.0 || (x.hi == 0.0 && x.lo < 0.0) ? -x : x; }
MRRR_HD bool dd_isfinite(const dd& x) { return isfinite(x.hi) && isfinite(x.lo); }

// square root: one Newton correction of the double root (Karp-Markstein form)
MRRR_HD dd dd_sqrt(const dd& a) {
    if (a.hi <= 0.0) return dd(0.0);
    double x = sqrt(a.hi);
    dd xx = two_prod(x, x);
    dd r = a - xx;
    return fast_two_sum(x, r.hi / (2.0 * x));
}

}  // namespace mrrr
