// The steps of Algorithm 1 as per-matrix / per-block / per-item functions.
// Each CUDA kernel of the solver is a thin wrapper that maps one thread to
// one call of a function below.
#pragma once

#include "mrrr_core.cuh"
#include "mrrr_fast.cuh"
#include "mrrr_types.cuh"

#include <cstring>
#include <type_traits>

#if defined(__CUDA_ARCH__)
#define MRRR_ATOMIC_ADD(p, v) atomicAdd((p), (v))
#define MRRR_ATOMIC_MAX(p, v) atomicMax((p), (v))
#else
template <class T> static inline T mrrr_host_add(T* p, T v) { T o = *p; *p += v; return o; }
template <class T> static inline T mrrr_host_max(T* p, T v) { T o = *p; if (v > *p) *p = v; return o; }
#define MRRR_ATOMIC_ADD(p, v) mrrr_host_add((p), (v))
#define MRRR_ATOMIC_MAX(p, v) mrrr_host_max((p), (v))
#endif

namespace mrrr {

template <class X> MRRR_HD double ld_x(const void* p, int i) { return (double)((const X*)p)[i]; }

// --------------------------------------------------------------- a1: scale + split

// Preprocessing (Sec. 2 "Preprocessing", Sec. 3.2 "Preprocessing"): scale T
// by a power of two so that ||T||_1 lies in [1/2, 1) (exact), set e_i = 0
// where |e_i| <= eps_x ||T||_1 (||T|| of the unreduced input), and record the
// irreducible blocks.
template <class X>
MRRR_HD void prep_matrix(MatrixDesc& M, BlockDesc* blocks, double* wd, double* we, const SolveCfg& cfg) {
    const int n = M.n;
    double tn = 0.0;
    bool finite = true;
    for (int i = 0; i < n; ++i) {
        double di = ld_x<X>(M.d, i);
        double s = fabs(di);
        if (!isfinite(di)) finite = false;
        if (i > 0) s += fabs(ld_x<X>(M.e, i - 1));
        if (i < n - 1) {
            double ei = ld_x<X>(M.e, i);
            if (!isfinite(ei)) finite = false;
            s += fabs(ei);
        }
        tn = fmax(tn, s);
    }
    if (!finite || !isfinite(tn)) {
        M.status = ST_ERR_NONFINITE;
        M.nblocks = 0;
        return;
    }
    double scale = 1.0;
    if (tn > 0.0) {
        int ex;
        frexp(tn, &ex);  // tn = m 2^ex, m in [1/2, 1)
        scale = ldexp(1.0, -ex);
    }
    M.scale = scale;
    M.tnorm = tn;
    const double thresh = cfg.eps_x * tn;
    int nb = 0;
    int start = 0;
    for (int i = 0; i < n; ++i) {
        wd[M.row0 + i] = ld_x<X>(M.d, i) * scale;
        bool end = (i == n - 1);
        if (i < n - 1) {
            double ei = ld_x<X>(M.e, i);
            if (fabs(ei) <= thresh) {
                ei = 0.0;
                end = true;
            }
            we[M.row0 + i] = ei * scale;
        } else {
            we[M.row0 + i] = 0.0;
        }
        if (end) {
            BlockDesc& B = blocks[M.row0 + nb];
            B.matrix = -1;  // set by the caller's matrix index
            B.row0 = M.row0 + start;
            B.mrow = start;
            B.n = i - start + 1;
            ++nb;
            start = i + 1;
        }
    }
    M.nblocks = nb;
}

// --------------------------------------------------------------- a2: root representation

// Root representation (Algorithm 1, lines 1-2): Gershgorin interval, a shift
// mu just outside one end so that T - mu I is definite (Sec. 3.2: a root
// representation is always found "by making T - mu I definite"), LDL^T in
// working precision, random relative perturbation, derived LD and LLD, and a
// rounded low-precision copy for the pre-bisection.  Split into steps so a
// CTA can run the two candidate factorizations on two warps and the
// element-wise work on all its threads.

// Step 1: Gershgorin bounds, pivmin, spectral diameter.  The bounds of the
// rows i0, i0 + stride, ... of the block are folded
// into *gl / *gu, and the largest e_i^2 into *emax2 (min and max are exact,
// so any split over threads gives the serial result).
MRRR_HD void root_bounds_part(const BlockDesc& B, const double* wd, const double* we, int i0, int stride, double* gl,
                              double* gu, double* emax2) {
    const int n = B.n;
    const double* a = wd + B.row0;
    const double* b = we + B.row0;
    for (int i = i0; i < n; i += stride) {
        double r = 0.0;
        if (i > 0) r += fabs(b[i - 1]);
        if (i < n - 1) {
            r += fabs(b[i]);
            *emax2 = fmax(*emax2, b[i] * b[i]);
        }
        *gl = fmin(*gl, a[i] - r);
        *gu = fmax(*gu, a[i] + r);
    }
}

template <class Y>
MRRR_HD void root_bounds_finish(BlockDesc& B, double gl, double gu, double emax2) {
    // 4x the smallest normal of the working precision keeps every reciprocal
    // of a guarded pivot finite
    B.pivmin = 4.0 * Prec<Y>::tiny * fmax(1.0, emax2);
    B.spdiam = gu - gl;
}

// Step 1 on one thread.
template <class Y>
MRRR_HD void root_bounds(BlockDesc& B, const double* wd, const double* we, double* gl_out, double* gu_out) {
    double gl = INFINITY, gu = -INFINITY, emax2 = 0.0;
    root_bounds_part(B, wd, we, 0, 1, &gl, &gu, &emax2);
    root_bounds_finish<Y>(B, gl, gu, emax2);
    *gl_out = gl;
    *gu_out = gu;
}

// Step 2 (one thread per side): factor T - mu I with mu = gl - delta (side 0,
// positive definite, into the D/L slots) or mu = gu + delta (side 1,
// negative definite, into the LD/LLD slots), growing delta until definite.
template <class Y>
MRRR_HD double root_candidate(const BlockDesc& B, const double* wd, const double* we, Y* reps, double gl,
                              double gu, int side, double* mu_out) {
    const int n = B.n;
    Y* rep = reps + 4 * (size_t)B.row0 + (side ? 2 * (size_t)n : 0);
    double bnd = fmax(fabs(gl), fabs(gu));
    double delta = 4.0 * n * 1.1102230246251565e-16 * bnd + 4.0 * B.pivmin;
    for (int attempt = 0; attempt < 40; ++attempt) {
        double mu = side ? gu + delta : gl - delta;
        double g;
#if defined(__CUDA_ARCH__)
        if constexpr (std::is_same<Y, double>::value) {
            g = ldl_factor_fast(wd + B.row0, we + B.row0, n, mu, side ? -1 : +1, rep);
        } else if constexpr (std::is_same<Y, dd>::value) {
            // double-double root: the factorization in binary64, widened
            // exactly.  The random relative perturbation of size xi = 4 eps_x
            // that follows (root_element) is as large as the rounding of a
            // binary64 factorization, so the root is still T - mu I perturbed
            // element-wise by O(eps_x) -- at the latency of binary64 instead of
            // a serial chain of double-double divisions.  The factorization is
            // written as binary64 into the first 2n words of this side's
            // region and widened in place from the top down (double-double
            // entry i covers binary64 words 2i, 2i+1 >= i).
            double* tmp = (double*)rep;
            g = ldl_factor_fast(wd + B.row0, we + B.row0, n, mu, side ? -1 : +1, tmp);
            if (g < INFINITY)
                for (int i = 2 * n - 1; i >= 0; --i) rep[i] = dd(tmp[i]);
        } else
#endif
            g = ldl_factor<Y>(wd + B.row0, we + B.row0, n, mu, side ? -1 : +1, rep);
        if (g < INFINITY) {
            *mu_out = mu;
            return g;
        }
        delta *= 16.0;
    }
    *mu_out = side ? gu + delta : gl - delta;
    return INFINITY;
}

// Step 3 (one thread): choose the side with the smaller growth, set mu, the
// bracket of the root spectrum, and the perturbation bound.
MRRR_HD void root_choose(BlockDesc& B, const MatrixDesc& M, double gl, double gu, double gL, double muL, double gR,
                         double muR, const SolveCfg& cfg) {
    const int n = B.n;
    bool right = !(gL <= gR) && gR < INFINITY;
    if (!(gL < INFINITY) && !(gR < INFINITY)) right = false;  // cannot happen for finite scaled input
    B.side = right ? -1 : +1;
    B.mu = right ? muR : muL;
    B.growth = right ? gR : gL;
    // xi is capped at eps_x n / 8 so that for tiny matrices the perturbation
    // alone cannot exceed the accuracy target 2 n eps_x ||T||
    double xi = fmin(cfg.xi, cfg.eps_x * (double)M.n / 8.0);
    double lo = gl - B.mu, hi = gu - B.mu;
    double pad = (4.0 * xi + 8.0 * n * cfg.eps_y) * fmax(fabs(lo), fabs(hi)) + 4.0 * B.pivmin;
    B.gl = lo - pad;
    B.gu = hi + pad;
}

// Step 4 (element i, after step 3): move the right-end candidate into place.
template <class Y>
MRRR_HD void root_move(const BlockDesc& B, Y* reps, int i) {
    if (B.side > 0) return;
    const int n = B.n;
    Y* rep = reps + 4 * (size_t)B.row0;
    rep[i] = rep[2 * n + i];
    if (i < n - 1) rep[n + i] = rep[3 * n + i];
}

// Step 5 (element i, after step 4): multiply d_i and l_i by (1 + xi r) with r
// uniform in [-1, 1) from the counter-based generator (Algorithm 1, line 2;
// Sec. 3.2, "Random perturbations"), form LD_i, LLD_i and the low copy.  The
// counter is keyed by the row within the matrix, so a matrix is perturbed
// identically alone and inside a batch.
template <class Y, class Lo>
MRRR_HD void root_element(const BlockDesc& B, const MatrixDesc& M, Y* reps, Lo* reps_lo, int i,
                          const SolveCfg& cfg, const double* we) {
    const int n = B.n;
    Y* rep = reps + 4 * (size_t)B.row0;
    Lo* lo = reps_lo + 2 * (size_t)B.row0;
    double xi = fmin(cfg.xi, cfg.eps_x * (double)M.n / 8.0);
    uint64_t c0 = 4ULL * (uint64_t)B.mrow + 2ULL * (uint64_t)i;
    Y d = rep[i];
    Y l = (i < n - 1) ? rep[n + i] : from_d<Y>(0.0);
    Y ld, lld;
    if (cfg.flags & MRRR_FLAG_E_REP) {
        // e-representation (Sec. 3.2, "Choice of representations"): the data
        // are d_i and the off-diagonal e_i of T - mu I itself (the scaled
        // input), perturbed by the same relative amounts; l_i = e_i / d_i
        Y e = (i < n - 1) ? from_d<Y>(we[B.row0 + i]) : from_d<Y>(0.0);
        if (xi > 0.0) {
            d = d + d * from_d<Y>(xi * sym_uniform(cfg.seed, c0));
            if (i < n - 1) e = e + e * from_d<Y>(xi * sym_uniform(cfg.seed, c0 + 1ULL));
        }
        l = (i < n - 1) ? e / d : from_d<Y>(0.0);
        ld = e;
        lld = e * l;
    } else {
        if (xi > 0.0) {
            d = d + d * from_d<Y>(xi * sym_uniform(cfg.seed, c0));
            if (i < n - 1) l = l + l * from_d<Y>(xi * sym_uniform(cfg.seed, c0 + 1ULL));
        }
        ld = d * l;
        lld = ld * l;
    }
    rep[i] = d;
    if (i < n - 1) {
        rep[n + i] = l;
        rep[2 * n + i] = ld;
        rep[3 * n + i] = lld;
    } else {
        rep[2 * n - 1] = from_d<Y>(0.0);
        rep[3 * n - 1] = from_d<Y>(0.0);
        rep[4 * n - 1] = from_d<Y>(0.0);
    }
    lo[i] = (Lo)to_d(d);
    lo[n + i] = (Lo)to_d(lld);
}

// Step 6 (one thread, after step 5): which eigenvalues the block computes.
template <class Y>
MRRR_HD void root_range(BlockDesc& B, const MatrixDesc& M, const double* wd, const Y* reps) {
    const int n = B.n;
    const Y* rep = reps + 4 * (size_t)B.row0;
    int wlo = 1, whi = n;
    if (M.range == RANGE_INDEX && M.nblocks == 1) {
        wlo = M.il;
        whi = M.iu;
    } else if (M.range == RANGE_VALUE) {
        if (n == 1) {
            double lam = wd[B.row0];
            bool in = lam > M.vl * M.scale && lam <= M.vu * M.scale;
            wlo = 1;
            whi = in ? 1 : 0;
        } else {
            Y pm = from_d<Y>(B.pivmin);
            wlo = negcount<Y>(rep, rep + 3 * n, n, from_d<Y>(M.vl * M.scale - B.mu), pm) + 1;
            whi = negcount<Y>(rep, rep + 3 * n, n, from_d<Y>(M.vu * M.scale - B.mu), pm);
        }
    }
    B.w_lo = wlo;
    B.w_hi = whi;
    if (wlo > whi) {
        B.f_lo = 1;
        B.f_hi = 0;
    } else {
        B.f_lo = wlo > 1 ? wlo - 1 : 1;
        B.f_hi = whi < n ? whi + 1 : n;
    }
    B.nitems = B.f_hi >= B.f_lo ? B.f_hi - B.f_lo + 1 : 0;
}

// A block of size one: its eigenvalue is d_1 exactly (mu = d_1, rep = 0).
template <class Y, class Lo>
MRRR_HD void root_trivial(BlockDesc& B, const double* wd, Y* reps, Lo* reps_lo) {
    Y* rep = reps + 4 * (size_t)B.row0;
    Lo* lo = reps_lo + 2 * (size_t)B.row0;
    B.mu = wd[B.row0];
    B.side = +1;
    B.growth = 0.0;
    rep[0] = rep[1] = rep[2] = rep[3] = from_d<Y>(0.0);
    lo[0] = lo[1] = Lo(0);
    B.gl = 0.0;
    B.gu = 0.0;
}

// Item t of one block (after the host-side scan assigned item0).
template <class Y, class Lo>
MRRR_HD void init_item(const BlockDesc& B, int bidx, Item& I, int t, const Y* reps, const Lo* reps_lo) {
    I.j = B.f_lo + t;
    I.lo = B.gl;
    I.hi = B.gu;
    I.gapL = INFINITY;
    I.gapR = INFINITY;
    I.sig_hi = B.mu;
    I.sig_lo = 0.0;
    I.rep = reps + 4 * (size_t)B.row0;
    I.rep_lo = reps_lo + 2 * (size_t)B.row0;
    I.n = B.n;
    I.block = bidx;
    I.matrix = B.matrix;
    I.outcol = -1;
    I.depth = 0;
    I.kind = KIND_OPEN;
    I.wanted = (I.j >= B.w_lo && I.j <= B.w_hi) ? 1 : 0;  // refined by assign_col
    I.rep_up = nullptr;
    I.sig_up_hi = 0.0;
    I.sig_up_lo = 0.0;
    I.span_lo = 0.0;
    I.span_hi = 0.0;
    I.span_gapL = INFINITY;
    I.span_gapR = INFINITY;
    I.lam_hi = 0.0;
    I.lam_lo = 0.0;
    I.rqi_done = 0;
    I.rhint = -1;
}

// --------------------------------------------------------------- a3: bisection

// Relative separation of two neighbouring brackets (Sec. 2, reldist):
// reldist(A, B) >= gaptol for neighbouring brackets A < B, evaluated
// without a division (the denominator is >= 0); gaptol = -inf separates all.
MRRR_HD bool separated(const Item& A, const Item& B, double gaptol) {
    if (gaptol == -INFINITY) return true;
    double den = fmax(fmax(fabs(A.lo), fabs(A.hi)), fmax(fabs(B.lo), fabs(B.hi)));
    return (B.lo - A.hi) >= gaptol * den;
}

// Neighbouring items belong to the same group when they share a rep.
MRRR_HD bool same_group(const Item& A, const Item& B) { return A.rep == B.rep && A.block == B.block; }


// Precision of the rounded copy of a rep: binary32 for binary32/binary64
// reps, binary64 for double-double reps.
template <class Y> struct LowType { typedef float T; };
template <> struct LowType<dd> { typedef double T; };

template <class T> MRRR_HD T bmax(const T& a, const T& b) { return a < b ? b : a; }
template <class T> MRRR_HD T bmin(const T& a, const T& b) { return b < a ? b : a; }
MRRR_HD double babs(double x) { return fabs(x); }
MRRR_HD dd babs(const dd& x) { return dd_abs(x); }
MRRR_HD float babs(float x) { return fabsf(x); }

// Sturm count for bisection: the tuned projective counts on the device when
// FAST (binary64 and double-double; classification brackets and their
// verification), the guarded divide form otherwise.
template <class Y, bool FAST>
MRRR_HD int count_at(const Y* D, const Y* LLD, int n, Y tau, Y pm) {
#if defined(__CUDA_ARCH__)
    if constexpr (FAST && std::is_same<Y, double>::value) return negcount_fast(D, LLD, n, tau, pm);
    if constexpr (FAST && std::is_same<Y, dd>::value) return negcount_dd_fast(D, LLD, n, tau, pm);
#endif
    return negcount<Y>(D, LLD, n, tau, pm);
}

// Multisection: kMS lanes per item evaluate the count at kMS equispaced
// interior points of the same bracket in one sweep, so each sweep divides
// the bracket into kMS + 1 parts instead of two.  The sweeps are sequential
// in the row index, so this trades spare throughput for latency.  (Wider
// sweeps and points at equal ratios shorten the approximation but leave the
// RQI with brackets from which more eigenpairs need a third step; four
// equispaced points measured best overall.)
constexpr int kMS = 4;
MRRR_HD double ms_point(double lo, double hi, int q) { return lo + (hi - lo) / (kMS + 1) * (q + 1); }

// Bisection for eigenvalue j (1-based) of the rep on the bracket [lo, hi]
// (Algorithm 1, lines 3 and 16; Sec. 2, "Classification of the
// eigenvalues"): stop when hi - lo <= max(rtol max(|lo|, |hi|), 2 pivmin).
// Invariant: negcount(lo) < j <= negcount(hi).  With verify != 0 the
// invariant is first re-established by widening the bracket (brackets
// carried over from a parent rep through a shift, whose eigenvalues differ
// from the parent's by the mixed relative perturbation of the shift).
// The bracket type Bt is double for classification and the working
// precision for the bisection fallback of the RQI.  Returns qd steps.
template <class Y, class Bt, bool FAST = false>
MRRR_HD unsigned long long bisect_bracket(const Y* rep, int n, int j, Bt& lo, Bt& hi, double pivmin, double rtol,
                                          int verify, int max_steps) {
    const Y* D = rep;
    const Y* LLD = rep + 3 * n;
    Y pm = from_d<Y>(pivmin);
    unsigned long long steps = 0;
    if (verify) {
        for (int side = 0; side < 2; ++side) {
            Bt w = bmax(hi - lo, Bt(4.0 * Prec<double>::eps) * bmax(babs(lo), babs(hi)));
            w = bmax(w, Bt(4.0 * pivmin));
            for (int it = 0; it < 200; ++it) {
                ++steps;
                if (side == 0) {
                    if (count_at<Y, FAST>(D, LLD, n, Y(lo), pm) < j) break;
                    lo = lo - w;
                } else {
                    if (count_at<Y, FAST>(D, LLD, n, Y(hi), pm) >= j) break;
                    hi = hi + w;
                }
                w = w + w;
            }
        }
    }
    for (int it = 0; it < max_steps; ++it) {
        Bt width = hi - lo;
        Bt tol = bmax(Bt(rtol) * bmax(babs(lo), babs(hi)), Bt(2.0 * pivmin));
        if (!(tol < width)) break;
        Bt mid = (lo + hi) * Bt(0.5);
        if (!(lo < mid && mid < hi)) break;
        ++steps;
        if (count_at<Y, FAST>(D, LLD, n, Y(mid), pm) >= j) hi = mid;
        else lo = mid;
    }
    return steps * (unsigned long long)n;
}

template <class Y>
MRRR_HD void bisect_item(Item& I, double pivmin, double rtol, int verify, int max_steps,
                         unsigned long long* steps_out) {
    if (I.n == 1) {
        I.lo = 0.0;
        I.hi = 0.0;
        return;
    }
    double lo = I.lo, hi = I.hi;
    unsigned long long s =
        bisect_bracket<Y, double, true>((const Y*)I.rep, I.n, I.j, lo, hi, pivmin, rtol, verify, max_steps);
    I.lo = lo;
    I.hi = hi;
    if (steps_out) *steps_out += s;
}

// Pre-bisection in the low precision on the rounded copy of the rep (Sec.
// 3.2, "Arithmetic used to approximate eigenvalues": bisection on a copy M_x
// in faster arithmetic), down to relative width `wrel`.  Nothing is trusted
// yet: verify_endpoint re-checks both ends in the working precision.
template <class Lo>
MRRR_HD unsigned long long bisect_lo_item(Item& I, double pivmin, double wrel, int max_steps) {
    const int n = I.n;
    if (n == 1) return 0;
    const Lo* D = (const Lo*)I.rep_lo;
    const Lo* LLD = D + n;
    Lo pm = (Lo)fmax(pivmin, (double)Prec<Lo>::tiny * 4.0);
    double lo = I.lo, hi = I.hi;
    unsigned long long steps = 0;
    for (int it = 0; it < max_steps; ++it) {
        if (!(hi - lo > wrel * fmax(fabs(lo), fabs(hi)))) break;
        double mid = 0.5 * (lo + hi);
        Lo m = (Lo)mid;
        if (!((double)m > lo && (double)m < hi)) break;  // no representable point inside
        ++steps;
        if (negcount_lo<Lo>(D, LLD, n, m, pm) >= I.j) hi = (double)m;
        else lo = (double)m;
    }
    I.lo = lo;
    I.hi = hi;
    return steps * (unsigned long long)n;
}

// Re-establish one end of the bracket in the working precision: side 0 needs
// negcount(lo) < j, side 1 needs negcount(hi) >= j.  A failing end is moved
// outward by a doubling step; after 8 failures it jumps to the bound of the
// whole root spectrum in the item's coordinates.  The check is split so a
// kernel can make the first count for every end and widen only the few that
// failed, densely packed: endpoint_ok (one count), endpoint_step (the first
// widening step, from the bracket before any end moved) and widen_endpoint
// (the loop after a failed first count).

template <class Y>
MRRR_HD int endpoint_count(const Item& I, const BlockDesc& B, int side) {
    const int n = I.n;
    const Y* rep = (const Y*)I.rep;
    return count_at<Y, true>(rep, rep + 3 * n, n, from_d<Y>(side ? I.hi : I.lo), from_d<Y>(B.pivmin));
}

MRRR_HD bool endpoint_holds(const Item& I, int side, int c) { return side ? (c >= I.j) : (c < I.j); }

template <class Y>
MRRR_HD bool endpoint_ok(const Item& I, const BlockDesc& B, int side) {
    if (I.n == 1) return true;
    return endpoint_holds(I, side, endpoint_count<Y>(I, B, side));
}

MRRR_HD double endpoint_step(const Item& I, const BlockDesc& B, int side) {
    double x = side ? I.hi : I.lo;
    return fmax(fmax(I.hi - I.lo, 4.0 * Prec<double>::eps * fabs(x)), 4.0 * B.pivmin);
}

// Returns the new end; *steps += qd steps, *fails += widenings (the failed
// first count included).
template <class Y>
MRRR_HD double widen_endpoint(const Item& I, const BlockDesc& B, int side, double w, unsigned long long* steps,
                              int* fails) {
    const int n = I.n;
    const Y* rep = (const Y*)I.rep;
    const Y* D = rep;
    const Y* LLD = rep + 3 * n;
    Y pm = from_d<Y>(B.pivmin);
    double x = side ? I.hi : I.lo;
    int f = 1;
    x = side ? x + w : x - w;
    w *= 2.0;
    unsigned long long st = 0;
    for (int it = 1; it < 64; ++it) {
        ++st;
        int c = count_at<Y, true>(D, LLD, n, from_d<Y>(x), pm);
        bool ok = side ? (c >= I.j) : (c < I.j);
        if (ok) break;
        ++f;
        if (f > 8) {
            // shift of this rep relative to the root: sigma - mu
            double off = (I.sig_hi - B.mu) + I.sig_lo;
            double pad = 4.0 * Prec<double>::eps * (fabs(B.gl) + fabs(B.gu) + fabs(off)) + 4.0 * B.pivmin;
            double bound = side ? (B.gu - off + pad) : (B.gl - off - pad);
            if (side ? (bound > x) : (bound < x)) {
                x = bound;
                continue;
            }
        }
        x = side ? x + w : x - w;
        w *= 2.0;
    }
    *steps += st * (unsigned long long)n;
    *fails += f;
    return x;
}

// Both steps for one end on one thread.  Returns qd steps; *fails counts
// the widenings.
template <class Y>
MRRR_HD unsigned long long verify_endpoint(Item& I, const BlockDesc& B, int side, int* fails) {
    if (I.n == 1) return 0;
    unsigned long long steps = (unsigned long long)I.n;
    if (endpoint_ok<Y>(I, B, side)) return steps;
    double x = widen_endpoint<Y>(I, B, side, endpoint_step(I, B, side), &steps, fails);
    if (side) I.hi = x;
    else I.lo = x;
    return steps;
}

// An item is certified when, for each neighbour in the same rep, the
// verified brackets already give reldist >= gaptol (Sec. 2 notes that the
// relative-accuracy requirement can be relaxed for eigenvalues with a large
// gap); such items skip the working-precision refinement.  Neighbours in
// another rep lie outside the current cluster and were separated by gaptol
// one level up.
MRRR_HD bool certified(int t, const Item* items, int count_all, double gaptol) {
    const Item& I = items[t];
    if (t > 0 && same_group(items[t - 1], I) && !separated(items[t - 1], I, gaptol)) return false;
    if (t + 1 < count_all && same_group(I, items[t + 1]) && !separated(I, items[t + 1], gaptol)) return false;
    return true;
}

// --------------------------------------------------------------- output columns

// Output column of item t: position of its eigenvalue among the wanted
// eigenvalues of its matrix.  One block: j - w_lo.  Several blocks: the rank
// by (value, block, j), with ties between blocks broken by block order.
MRRR_HD void assign_col(int t, Item* items, const MatrixDesc* mats, const BlockDesc* blocks) {
    Item& I = items[t];
    const MatrixDesc& M = mats[I.matrix];
    const BlockDesc& B = blocks[I.block];
    if (M.nblocks == 1) {
        I.outcol = I.wanted ? I.j - B.w_lo : -1;
        return;
    }
    double key = 0.5 * (I.lo + I.hi) + B.mu;
    int rank = 0;
    for (int u = M.item0; u < M.item0 + M.nitems; ++u) {
        if (u == t) continue;
        const Item& U = items[u];
        if (M.range != RANGE_INDEX && !U.wanted) continue;
        double k2 = 0.5 * (U.lo + U.hi) + blocks[U.block].mu;
        if (k2 < key || (k2 == key && (U.block < I.block || (U.block == I.block && U.j < I.j)))) ++rank;
    }
    if (M.range == RANGE_INDEX) {
        bool want = (rank + 1 >= M.il) && (rank + 1 <= M.iu);
        I.wanted = want ? 1 : 0;
        I.outcol = want ? rank - (M.il - 1) : -1;
    } else {
        I.outcol = I.wanted ? rank : -1;
    }
}

// --------------------------------------------------------------- a4: classification


// Partition (Algorithm 1, line 7), one thread per item: j and j+1 of the
// same rep are separated when reldist(j, j+1) >= gaptol (Sec. 2,
// "Classification of the eigenvalues").  The first item of every run acts:
// a run of one is a singleton (gaps recorded, appended to the singleton list
// if wanted); a longer run with a wanted member becomes a cluster (appended
// with its members and its outer gaps).  Other threads only read neighbours'
// brackets, so the partition is race-free.
MRRR_HD void classify_item(int t, Item* items, int K, double gaptol, int* single_list, Cluster* clusters,
                           int* member_list, DevCounters* C) {
    Item& I = items[t];
    bool has_l = t > 0 && same_group(items[t - 1], I);
    bool has_r = t + 1 < K && same_group(I, items[t + 1]);
    if (has_l && !separated(items[t - 1], I, gaptol)) return;  // inside a run
    bool cut_r = !has_r || separated(I, items[t + 1], gaptol);
    if (cut_r) {
        double mid = 0.5 * (I.lo + I.hi);
        if (has_l) I.gapL = mid - items[t - 1].hi;
        if (has_r) I.gapR = items[t + 1].lo - mid;
        if (I.wanted) {
            I.kind = KIND_SINGLETON;
            int slot = MRRR_ATOMIC_ADD(&C->nsingle, 1);
            single_list[slot] = t;
        } else {
            I.kind = KIND_DROPPED;
        }
        return;
    }
    int e = t + 1;
    while (e + 1 <= K - 1 && same_group(items[e], items[e + 1]) && !separated(items[e], items[e + 1], gaptol)) ++e;
    ++e;  // run [t, e)
    bool has_e = e < K && same_group(items[e - 1], items[e]);
    double gL = has_l ? I.lo - items[t - 1].hi : I.gapL;
    double gR = has_e ? items[e].lo - items[e - 1].hi : items[e - 1].gapR;
    int any = 0;
    for (int u = t; u < e; ++u) any |= items[u].wanted;
    if (!any) {
        for (int u = t; u < e; ++u) items[u].kind = KIND_DROPPED;
        return;
    }
    int c = MRRR_ATOMIC_ADD(&C->ncluster, 1);
    int m0 = MRRR_ATOMIC_ADD(&C->nmember, e - t);
    // a cluster whose rep is itself a child gets a second slot, for the
    // alternative parent rep of backtracking (shift_cluster)
    const unsigned long long slots = I.rep_up ? 2ULL : 1ULL;
    unsigned long long off = MRRR_ATOMIC_ADD(&C->pool_need, slots * 4ULL * (unsigned long long)I.n);
    Cluster& Kc = clusters[c];
    Kc.a = t;
    Kc.b = e;
    Kc.n = I.n;
    Kc.pool_off = (long long)off;
    Kc.gapL = gL;
    Kc.gapR = gR;
    Kc.depth = I.depth;
    for (int u = t; u < e; ++u) {
        items[u].kind = KIND_CLUSTER;
        member_list[m0 + (u - t)] = u;
    }
    items[t].gapL = gL;
    items[e - 1].gapR = gR;
    MRRR_ATOMIC_MAX(&C->largest_cluster, e - t);
    MRRR_ATOMIC_ADD(&C->nclusters_total, 1);
}

// --------------------------------------------------------------- a5: cluster -> child rep

// Growth of the child at shift tau as seen by an approximate eigenvector of
// the cluster: sum_i |d+_i| z_i^2 / ||z||^2, with z the twisted-factorization
// vector of the parent at tau (tau lies next to the cluster, so z is
// dominated by the cluster's invariant subspace).  This weighs the element
// growth by the vector it acts on, as conditional element growth does
// (Definition "Conditional element growth", Sec. 2): a large pivot where the
// eigenvector is negligible does no harm.
//
// *kappa receives the relative condition number of the child's eigenvalue
// along the same vector, the quantity relative robustness bounds (k_rr,
// Definition of an RRR, Sec. 2): with y = L+^T z,
//     kappa = sum_i |d+_i| y_i^2 / | sum_i d+_i y_i^2 |,
// the relative change of the Rayleigh quotient z^T L+ D+ L+^T z under
// element-wise relative perturbations of the d+_i (one for a definite
// child).  Uses `work` (3n words).
template <class Y>
MRRR_HD double weighted_growth(const Y* parent, int n, Y tau, Y pm, Y* work, double* kappa = nullptr) {
    Scratch<Y> Wk;
    Wk.a = work;
    Wk.b = work + n;
    Wk.stride = 1;
    Y gamma;
    TwistResult<Y> tr = twisted_solve<Y>(parent, n, tau, pm, Wk, &gamma);
    double nrm2 = to_d(tr.nrm2);
    RepPtr<Y> P(parent, n);
    Y s = -tau;
    double acc = 0.0, absq = 0.0, q = 0.0;
    for (int i = 0; i < n; ++i) {
        Y dp = P.D[i] + s;
        if (ysmall(dp, pm)) dp = -pm;
        double z = to_d(work[i]);
        acc += fabs(to_d(dp)) * z * z;
        if (i < n - 1) {
            const Y lp = qdiv<Y>(P.LD[i], dp);
            const double y = z + to_d(lp) * to_d(work[i + 1]);
            absq += fabs(to_d(dp)) * y * y;
            q += to_d(dp) * y * y;
            s = lp * P.L[i] * s - tau;
        } else {
            absq += fabs(to_d(dp)) * z * z;
            q += to_d(dp) * z * z;
        }
    }
    if (kappa) {
        const double k = absq / fabs(q);
        *kappa = isfinite(k) ? k : INFINITY;
    }
    double r = acc / nrm2;
    return isfinite(r) ? r : INFINITY;
}

// Child rep parent - tau I and its rounded low-precision copy; returns the
// element growth.  The device binary64 path builds both in one pass.
template <class Y, class Lo>
MRRR_HD double child_transform(const Y* parent, int n, Y tau, Y pm, Y* out, Lo* out_lo, bool erep) {
#if defined(__CUDA_ARCH__)
    if constexpr (std::is_same<Y, double>::value && std::is_same<Lo, float>::value)
        return dstqds_fast(parent, n, tau, to_d(pm), out, out_lo, erep);
#endif
    double g = dstqds<Y>(parent, n, tau, pm, out, erep);
    if (out) {
        for (int i = 0; i < n; ++i) {
            out_lo[i] = (Lo)to_d(out[i]);
            out_lo[n + i] = (Lo)to_d(out[3 * n + i]);
        }
    }
    return g;
}

// New RRR for a cluster (Algorithm 1, lines 15-17): a shift tau just outside
// the left or right end of the cluster, child = parent - tau I by the
// stationary transform in working precision.  Candidates back off from the
// cluster by a growing distance, never beyond half the gap to the rest of
// the spectrum (Sec. 3.2: a small gaptol leaves room to back off).  A
// candidate is accepted when the element growth max |d+_i|, or else the
// growth weighted by an approximate cluster vector, is at most
// growth_k * spdiam(root).  In mixed precision the plain growth test uses
// the relaxed bound of Eq. (3.6); MRRR_FLAG_RRR_TEST adds the relative
// robustness test with the k_rr bound of Eq. (3.7).
//
// Backtracking (Sec. 3.2, "The representation tree": a cluster whose
// candidates all fail can be processed again "by choosing different shifts
// at a higher level of the tree"): when no candidate built from the parent
// P passes and P is itself a child -- made from its own parent G for a
// cluster spanning [span_lo, span_hi] of G -- the candidate search for that
// cluster is run again from G, skipping the shift that made P, and gives an
// alternative parent P' (kept in a second pool slot of this cluster); the
// cluster's members move to P' and the search for their child runs there.
// If that fails too, the candidate with the smallest weighted growth of the
// searches is taken and counted in reps_failed.
//
// Members move to the child: rep (and its low-precision copy), sigma +=
// tau, brackets shifted into the child's coordinates (re-verified by the
// refinement that follows).
template <class Y, class Lo>
MRRR_HD void shift_cluster(const Cluster& K, Item* items, const BlockDesc* blocks, Y* pool, Lo* pool_lo,
                           const SolveCfg& cfg, DevCounters* C) {
    const int n = K.n;
    Item& first = items[K.a];
    Item& last = items[K.b - 1];
    const BlockDesc& B = blocks[first.block];
    Y pm = from_d<Y>(B.pivmin);
    Y* child = pool + K.pool_off;
    Lo* child_lo = pool_lo + K.pool_off / 2;
    const double bound = cfg.growth_k * B.spdiam;
    // Sec. 3.2, Eq. (3.6): with y > x the element growth may reach
    // max{10, eps_x / (eps_y sqrt(n))} spdiam without loss of accuracy
    const double relaxed = (cfg.mixed && !(cfg.flags & MRRR_FLAG_STRICT_GROWTH))
                               ? fmax(cfg.growth_k, cfg.eps_x / (cfg.eps_y * sqrt((double)n))) * B.spdiam
                               : bound;
    unsigned long long steps = 0;
    const bool erep = (cfg.flags & MRRR_FLAG_E_REP) != 0;
    // relative robustness (Sec. 3.2, Eq. (3.7)): with y > x the constant may
    // reach max{10, eps_x gaptol / (eps_y sqrt(n))} without loss of accuracy
    const bool rrtest = (cfg.flags & MRRR_FLAG_RRR_TEST) != 0;
    const double krr_bound = (cfg.mixed && !(cfg.flags & MRRR_FLAG_STRICT_GROWTH))
                                 ? fmax(10.0, cfg.eps_x * cfg.gaptol / (cfg.eps_y * sqrt((double)n)))
                                 : 10.0;
    struct Found {
        bool accepted;
        bool relaxed_only;
        double tau, w;
        double stored;  // the candidate whose rep is in the output slot (NaN: none)
        double kappa;   // relative condition estimate of the accepted candidate (-1: not measured)
    };
    // candidate search from `parent` for a cluster spanning [lo, hi] in its
    // coordinates with bracket width bw; the candidate reps are built into
    // `out` (which doubles as work space); `reject` turns every acceptance
    // down (test hook); the candidate `skip` is not tried
    auto search = [&](const Y* parent, double lo, double hi, double bw, double gapL, double gapR, Y* out, Lo* out_lo,
                      bool reject, double skip) {
        const double span = hi - lo;
        double base = fmax(fmax(0.25 * span, 2.0 * bw), 4.0 * cfg.eps_y * fmax(fabs(lo), fabs(hi)));
        base = fmax(base, 4.0 * B.pivmin);
        Found f{false, false, lo - base, INFINITY, NAN, -1.0};
        for (int k = 0; k < 6 && !f.accepted; ++k) {
            double delta = base * (double)(1 << k);
            for (int side = 0; side < 2 && !f.accepted; ++side) {
                double gap = side == 0 ? gapL : gapR;
                if (k > 0 && delta > 0.5 * gap) continue;
                double tau = side == 0 ? lo - delta : hi + delta;
                if (tau == skip) continue;
                // the first candidate is usually accepted: build it in place
                bool store = !(f.stored == f.stored);
                double g = child_transform<Y, Lo>(parent, n, from_d<Y>(tau), pm, store ? out : (Y*)nullptr,
                                                  out_lo, erep);
                f.stored = store ? tau : f.stored;
                steps += n;
                if (!reject && !rrtest && g <= relaxed) {
                    f.tau = tau;
                    f.accepted = true;
                    f.relaxed_only = g > bound;
                    break;
                }
                double kappa = 0.0;
                double w = weighted_growth<Y>(parent, n, from_d<Y>(tau), pm, out, &kappa);
                f.stored = NAN;
                steps += 3ULL * n;
                const bool rr_ok = !rrtest || kappa <= krr_bound;
                if (!reject && rr_ok && (g <= relaxed || w <= bound)) {
                    f.tau = tau;
                    f.accepted = true;
                    f.relaxed_only = g > bound && w > bound;
                    f.kappa = kappa;
                    break;
                }
                if (w < f.w) {
                    f.w = w;
                    f.tau = tau;
                }
            }
        }
        return f;
    };
    const double bw = fmax(first.hi - first.lo, last.hi - last.lo);
    const Y* parent = (const Y*)first.rep;
    dd sig_from = dd(first.sig_hi, first.sig_lo);
    const Y* from = parent;
    const void* from_up = first.rep_up;  // the parent's own parent (for the members' rep_up)
    dd sig_up = dd(first.sig_up_hi, first.sig_up_lo);
    double move = 0.0;  // shift of the members' brackets into the coordinates of `from`
    // test hook: turn down every candidate built from a parent that is itself
    // a child, so that the backtracking branch runs
    const bool hook = (cfg.flags & MRRR_FLAG_TEST_REJECT_CHILD) && first.rep_up != nullptr;
    // test hook: turn down every candidate (the "no suitable representation"
    // branch: the best failed candidate is taken)
    const bool no_rep = (cfg.flags & MRRR_FLAG_TEST_NO_REP) != 0;
    Found f = search(parent, first.lo, last.hi, bw, K.gapL, K.gapR, child, child_lo, hook || no_rep, NAN);
    if (!f.accepted && first.rep_up != nullptr) {
        // backtracking: another rep for the parent's cluster, from the
        // parent's parent G, skipping the shift that made the parent
        MRRR_ATOMIC_ADD(&C->reps_backtracked, 1);
        const Y* G = (const Y*)first.rep_up;
        const dd tp = dd(first.sig_hi, first.sig_lo) - sig_up;  // the shift that made P from G
        const double tau_p = tp.hi + tp.lo;
        Y* alt = child + 4 * (size_t)n;
        Lo* alt_lo = child_lo + 2 * (size_t)n;
        // the alternative parent depends on the parent's cluster alone (its
        // span and gaps in G, the skipped shift), not on this cluster: every
        // cluster of P that backtracks rebuilds the same P', so their vectors
        // share one representation and stay orthogonal to each other
        const double pw = 1e-3 * (first.span_hi - first.span_lo);
        Found fp = search(G, first.span_lo, first.span_hi, pw, first.span_gapL, first.span_gapR, alt, alt_lo, no_rep,
                          tau_p);
        if (!(fp.stored == fp.tau)) child_transform<Y, Lo>(G, n, from_d<Y>(fp.tau), pm, alt, alt_lo, erep);
        steps += n;
        if (!fp.accepted) MRRR_ATOMIC_ADD(&C->reps_failed, 1);
        // the members in the coordinates of P' = G - tau' I: + tau_p - tau'
        const double mv = tau_p - fp.tau;
        Found g = search(alt, first.lo + mv, last.hi + mv, bw, K.gapL, K.gapR, child, child_lo, no_rep, NAN);
        if (g.accepted || g.w < f.w) {
            f = g;
            from = alt;
            from_up = G;
            sig_from = sig_up + dd(fp.tau);
            move = mv;
            // P' is the members' new parent rep: it was made for the
            // parent's cluster, whose span stays the same in G
        }
        f.stored = NAN;  // `child` may hold a candidate of either search
    }
    if (!f.accepted) MRRR_ATOMIC_ADD(&C->reps_failed, 1);
    if (f.accepted && f.relaxed_only) MRRR_ATOMIC_ADD(&C->reps_relaxed, 1);
    if (f.kappa >= 0.0) {
        // largest relative condition estimate of an accepted child (the bit
        // patterns of non-negative doubles order like the values)
        unsigned long long kb;
        memcpy(&kb, &f.kappa, sizeof(kb));
        MRRR_ATOMIC_MAX(&C->krr_max_bits, kb);
        if (f.kappa > 10.0) MRRR_ATOMIC_ADD(&C->reps_krr_relaxed, 1);
    }
    if (!(f.stored == f.tau)) {
        child_transform<Y, Lo>(from, n, from_d<Y>(f.tau), pm, child, child_lo, erep);
        steps += n;
    }
    MRRR_ATOMIC_ADD(&C->qd_shift, steps);
    // sigma_child = sigma_from + tau, kept as an unevaluated double pair
    const dd sig = sig_from + dd(f.tau);
    const double span_lo = first.lo + move, span_hi = last.hi + move;  // this cluster, in `from`
    (void)from_up;
    for (int u = K.a; u < K.b; ++u) {
        Item& I = items[u];
        I.lo = I.lo + move - f.tau;
        I.hi = I.hi + move - f.tau;
        I.rep_up = from;
        I.sig_up_hi = sig_from.hi;
        I.sig_up_lo = sig_from.lo;
        I.span_lo = span_lo;
        I.span_hi = span_hi;
        I.span_gapL = K.gapL;
        I.span_gapR = K.gapR;
        I.rep = child;
        I.rep_lo = child_lo;
        I.sig_hi = sig.hi;
        I.sig_lo = sig.lo;
        I.depth = K.depth + 1;
        I.kind = KIND_OPEN;
    }
    MRRR_ATOMIC_MAX(&C->d_max, K.depth + 1);
}

// --------------------------------------------------------------- a6 + a7: RQI and store

// One twisted solve; on the device a binary64 solve with contiguous scratch
// uses the tuned transform, which also reports the arg-max of |z| (else
// *imax = -1) and can reuse a given twist index r_hint >= 0.
template <class Y>
MRRR_HD TwistResult<Y> twist_step(const Y* rep, int n, Y lam, Y pm, const Scratch<Y>& Wk, Y* gamma, int* imax,
                                  int r_hint) {
#if defined(__CUDA_ARCH__)
    if constexpr (std::is_same<Y, double>::value) {
        if (Wk.stride == 1) return twisted_solve_fast(rep, n, lam, to_d(pm), Wk.a, Wk.b, gamma, imax, r_hint);
    }
#endif
#if defined(__CUDA_ARCH__)
    if constexpr (std::is_same<Y, dd>::value) {
        if (Wk.stride == 1 && r_hint >= 0) return twisted_fixed_proj_dd(rep, n, lam, pm, Wk, gamma, imax, r_hint);
    }
#endif
    // double-double without a twist index, and the host build of binary64
    // (which follows the device's steps): the generic solve, at the given
    // twist index when there is one
    if constexpr (std::is_same<Y, dd>::value || std::is_same<Y, double>::value)
        return twisted_solve<Y>(rep, n, lam, pm, Wk, gamma, r_hint, imax);
    *imax = -1;
    return twisted_solve<Y>(rep, n, lam, pm, Wk, gamma);
}

// Rayleigh quotient iteration with twisted factorizations, guarded by
// bisection (Algorithm 1, line 10; Sec. 2, "Rayleigh quotient iteration"):
// each step solves at lambda, updates the bracket with the inertia of the
// stationary part, and corrects lambda by gamma_r / ||z||^2.  It stops when
// the residual |gamma_r| / ||z|| is below k_rs gap eps_x sqrt(n) (mixed,
// Sec. 3.2) or k_rs gap n eps / gaptol (plain, Eq. 2.2), or when the
// correction stagnates below 4 eps_y |lambda|.  If the correction leaves the
// bracket or the step budget runs out, lambda is bisected to relative
// accuracy eps_x sqrt(n) gaptol (mixed) / n eps (plain) and one twisted solve
// gives the vector (Sec. 3.2, "Rayleigh quotient iteration").  The vector is
// normalised, signed (largest entry positive), rounded to x and stored with
// lambda + sigma (Algorithm 1, line 11; Sec. 3.3).
//
// The iteration runs in passes of at most pass_iters steps: an eigenpair not
// converged at the end of a pass (and not in the final pass) saves its shift,
// bracket and twist index in I and returns false ("parked"), so that the few
// slow eigenpairs continue in a later, densely packed launch instead of
// holding a whole warp.  Returns true when the eigenpair was stored.  With
// store_scale != null (binary64 and binary32 working precision) the vector
// is left unnormalised in the scratch and the factor 1/||z|| (with the sign)
// is returned there for a warp-cooperative store.
template <class X, class Y>
MRRR_HD bool rqi_item(Item& I, MatrixDesc* mats, const BlockDesc* blocks, const SolveCfg& cfg,
                      const Scratch<Y>& Wk, DevCounters* C, int pass_iters, bool final_pass,
                      double* store_scale = nullptr) {
    typedef typename Acc<Y>::T A_t;
    MatrixDesc& M = mats[I.matrix];
    const BlockDesc& B = blocks[I.block];
    const int n = I.n;
    const Y* rep = (const Y*)I.rep;
    Y pm = from_d<Y>(B.pivmin);
    const double sq = sqrt((double)n);
    double gap = fmin(I.gapL, I.gapR);
    if (!(gap < INFINITY)) gap = fmax(B.spdiam, 1e-300);
    const double tol = cfg.mixed ? cfg.krs * gap * cfg.eps_x * sq : cfg.krs * gap * n * cfg.eps_y / cfg.gaptol;
    Y lo = from_d<Y>(I.lo), hi = from_d<Y>(I.hi);
    if (std::is_same<Y, double>::value && I.rqi_done == 0) {
        // the bracket was verified by the tuned binary64 count, which is exact
        // for the rep perturbed element-wise by a few ulps, so its eigenvalues
        // can sit ~n ulps |lambda| from the ones the steps below converge to
        // (rounded in another order).  Widen the safeguard by a generous
        // multiple of that so a correct Rayleigh correction near an end is not
        // rejected as leaving the bracket (the inertia of the first step
        // narrows it again).
        const double pad = 16.0 * n * 0x1p-44 * fmax(fabs(I.lo), fabs(I.hi)) + 4.0 * B.pivmin;
        lo = from_d<Y>(I.lo - pad);
        hi = from_d<Y>(I.hi + pad);
    }
    Y lam = (lo + hi) * from_d<Y>(0.5);
    if (I.rqi_done > 0) {  // continue from the saved shift
        if constexpr (std::is_same<Y, dd>::value) lam = dd(I.lam_hi, I.lam_lo);
        else lam = from_d<Y>(I.lam_hi);
    }
    if (I.rqi_done == 0 && pass_iters == 2 && !final_pass) {
        // first pass: predict whether two steps suffice.  Every step solves
        // with the right-hand side e_r, so the shift error contracts like
        // e -> c e^2 / gap (c ~ 1/2 to 2/3 measured) and the residual after
        // the next solve is ~10-20 e; an eigenpair whose e0 (half the
        // bracket) does not pass 20 e0^2 / gap <= tol gets its third step in
        // this pass rather than in a later, nearly empty launch
        const double e0 = 0.5 * (I.hi - I.lo);
        if (20.0 * e0 * e0 > tol * gap) pass_iters = 3;
    }
    Y gamma = from_d<Y>(0.0);
    TwistResult<Y> tr;
    Y lam_out = lam;
    bool conv = false;
    int iters = 0;
    int imax_t = -1;
    unsigned long long steps = 0, steps_low = 0;
    if (n == 1) {
        Wk.A(0) = from_d<Y>(1.0);
        tr.r = 0;
        tr.nrm2 = A_t(1.0);
        lam_out = from_d<Y>(0.0);
        conv = true;
    } else {
        // after the first step the twist index is the largest entry of the
        // previous iterate (one pass of the transforms instead of two); the
        // first step takes it from a low-precision sweep over the rounded
        // copy of the rep, so it too needs one working-precision pass
        int r_hint = I.rhint;
        // (where a fixed-r step exists: binary64 and double-double)
        if ((std::is_same<Y, double>::value || std::is_same<Y, dd>::value) && I.rqi_done == 0 && r_hint < 0 &&
            I.rep_lo != nullptr) {
            typedef typename LowType<Y>::T Lo;
            const Lo* Dl = (const Lo*)I.rep_lo;
#if defined(__CUDA_ARCH__)
            if constexpr (std::is_same<Lo, float>::value)
                r_hint = twist_index_lo_fast(Dl, Dl + n, n, (float)to_d(lam), (float*)Wk.a);
            else
#endif
                r_hint = twist_index_lo<Lo>(Dl, Dl + n, n, (Lo)to_d(lam), (Lo*)Wk.a);
            steps_low = 2ULL * n;
        }
        const int done0 = I.rqi_done;
        for (int it = 0; it < pass_iters && done0 + it < cfg.max_rqi; ++it) {
            const bool r_from_sweep = it == 0 && done0 == 0 && r_hint >= 0;
            tr = twist_step<Y>(rep, n, lam, pm, Wk, &gamma, &imax_t, r_hint);
            steps += (r_hint < 0 ? 2ULL : 1ULL) * n;
            r_hint = imax_t;
            ++iters;
            // a first step whose low-precision twist index missed the large
            // entries of the vector (z_r = 1 but some |z_i| > 4) gives a poor
            // Rayleigh correction: allow one step more in this pass rather than
            // parking the eigenpair for a nearly empty later launch
            if (r_from_sweep && !final_pass && imax_t >= 0 && pass_iters < 3 &&
                fabs(to_d(Wk.A(imax_t))) > 4.0)
                pass_iters = 3;
            if (tr.neg >= I.j) hi = bmin(hi, lam);
            else lo = bmax(lo, lam);
            double nrm2 = to_d(tr.nrm2);
            double resid = fabs(to_d(gamma)) / sqrt(nrm2);
            Y corr = gamma / Y(tr.nrm2);
            if (resid <= tol || fabs(to_d(corr)) <= 4.0 * cfg.eps_y * fabs(to_d(lam))) {
                lam_out = lam + corr;
                conv = true;
                break;
            }
            Y nl = lam + corr;
            // inside the bracket, or outside by no more than rounding: an end
            // can sit within rounding of the eigenvalue (a pre-bisection point
            // or an earlier iterate), and a correct step then lands a hair
            // beyond it; a neighbouring eigenvalue is a whole gap away
            const Y slack = from_d<Y>(16.0 * n * cfg.eps_y * fabs(to_d(lam)));
            const Y width = hi - lo;
            if (lo - slack < nl && nl < hi + slack) {
                lam = nl;
            } else if ((nl >= hi && nl - hi <= width * from_d<Y>(0.25)) ||
                       (nl <= lo && lo - nl <= width * from_d<Y>(0.25))) {
                // a short overshoot past an end that lies close to the
                // eigenvalue: step to just inside that end (the vector, and
                // so the twist index, stays good)
                lam = nl >= hi ? hi - width * from_d<Y>(0x1p-10) : lo + width * from_d<Y>(0x1p-10);
            } else {
                // the correction left the bracket (it points at another
                // eigenvalue): take a bisection step instead, with the bracket
                // just narrowed by the inertia at lam, and refactor fully
                lam = (lo + hi) * from_d<Y>(0.5);
                r_hint = -1;
                // from the bisected shift the iteration needs about two more
                // steps: take them in this pass
                if (!final_pass && pass_iters < it + 3) pass_iters = it + 3;
            }
        }
        if (!conv && !final_pass && done0 + iters < cfg.max_rqi) {
            // park: save the state, rounding the bracket outward to binary64
            double lod = to_d(lo), hid = to_d(hi);
            I.lo = nextafter(lod, -HUGE_VAL);
            I.hi = nextafter(hid, HUGE_VAL);
            if constexpr (std::is_same<Y, dd>::value) {
                I.lam_hi = lam.hi;
                I.lam_lo = lam.lo;
            } else {
                I.lam_hi = to_d(lam);
                I.lam_lo = 0.0;
            }
            I.rqi_done = done0 + iters;
            I.rhint = r_hint;
            MRRR_ATOMIC_ADD(&C->rqi_iters, iters);
            MRRR_ATOMIC_ADD(&C->rqi_rows, (unsigned long long)iters * (unsigned long long)n);
            MRRR_ATOMIC_ADD(&C->qd_rqi, steps);
            if (steps_low) MRRR_ATOMIC_ADD(&C->qd_steps_low, steps_low);
            return false;
        }
        if (!conv) {
            MRRR_ATOMIC_ADD(&C->fallbacks, 1);
            double rt = cfg.mixed ? cfg.eps_x * sq * cfg.gaptol : n * cfg.eps_y;
            rt = fmax(rt, 4.0 * cfg.eps_y);
            // bisection: first with the fast count, then the last bits with the
            // fully accurate one
            steps += bisect_bracket<Y, Y, true>(rep, n, I.j, lo, hi, B.pivmin, fmax(rt, 1e-12), 1, 600);
            steps += bisect_bracket<Y, Y>(rep, n, I.j, lo, hi, B.pivmin, rt, 1, 600);
            // then a few safeguarded RQI steps from the midpoint, which now
            // lies close enough for the iteration to settle
            lam = (lo + hi) * from_d<Y>(0.5);
            int rh = -1;
            for (int k = 0; k < 4; ++k) {
                tr = twist_step<Y>(rep, n, lam, pm, Wk, &gamma, &imax_t, rh);
                steps += (rh < 0 ? 2ULL : 1ULL) * n;
                rh = imax_t;
                ++iters;
                if (tr.neg >= I.j) hi = bmin(hi, lam);
                else lo = bmax(lo, lam);
                double nrm2 = to_d(tr.nrm2);
                double resid = fabs(to_d(gamma)) / sqrt(nrm2);
                Y corr = gamma / Y(tr.nrm2);
                lam_out = lam + corr;
                conv = resid <= fmax(tol, 8.0 * cfg.eps_y * n * fabs(to_d(lam))) ||
                       fabs(to_d(corr)) <= 4.0 * cfg.eps_y * fabs(to_d(lam));
                if (conv) break;
                Y nl = lam + corr;
                if (lo < nl && nl < hi) {
                    lam = nl;
                } else {
                    lam = (lo + hi) * from_d<Y>(0.5);
                    rh = -1;
                }
            }
            if (!conv) {
                MRRR_ATOMIC_ADD(&C->noconv, 1);
                M.status = ST_ERR_NOCONV;  // every writer stores the same value
            }
        }
    }
    MRRR_ATOMIC_ADD(&C->rqi_iters, iters);
    MRRR_ATOMIC_ADD(&C->rqi_rows, (unsigned long long)iters * (unsigned long long)n);
    MRRR_ATOMIC_ADD(&C->qd_rqi, steps);
    if (steps_low) MRRR_ATOMIC_ADD(&C->qd_steps_low, steps_low);
    // eigenvalue of T: (lambda + sigma) / scale
    dd lt = dd(to_d(lam_out)) + dd(I.sig_hi, I.sig_lo);
    if constexpr (std::is_same<Y, dd>::value) lt = lam_out + dd(I.sig_hi, I.sig_lo);
    double lam_T = (lt.hi + lt.lo) / M.scale;
    // normalise, fix the sign (largest entry positive), cast to x, store
    A_t nrm = ysqrt(tr.nrm2);
    int imax = imax_t;
    if (imax < 0) {
        imax = 0;
        double zmax = -1.0;
        for (int i = 0; i < n; ++i) {
            double z = fabs(to_d(Wk.A(i)));
            if (z > zmax) {
                zmax = z;
                imax = i;
            }
        }
    }
    double sgn = to_d(Wk.A(imax)) < 0.0 ? -1.0 : 1.0;
    X* Z = (X*)M.Z + (size_t)I.outcol * (size_t)M.ldz + B.mrow;
    if constexpr (std::is_same<A_t, dd>::value) {
        // double-double: divide in working precision, round once to x
        for (int i = 0; i < n; ++i) {
            A_t z = A_t(Wk.A(i)) / nrm;
            Z[i] = (X)(sgn * to_d(z));
        }
    } else {
        double inv = sgn / to_d(nrm);
        if (store_scale) {
            *store_scale = inv;  // the caller stores z * inv (coalesced across a warp)
        } else {
            for (int i = 0; i < n; ++i) Z[i] = (X)(to_d(Wk.A(i)) * inv);
        }
    }
    ((X*)M.W)[I.outcol] = (X)lam_T;
    return true;
}

}  // namespace mrrr
