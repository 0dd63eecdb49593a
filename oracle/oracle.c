/*
 * Oracle for the real symmetric tridiagonal eigenproblem T z = lambda z.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the solver library links, calls or
 * includes this file; only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load it (as liboracle.so through ctypes).
 * It shares no code, header, table or constant with the CUDA solver.
 *
 * Everything here is the plain textbook definition, carried out in IEEE
 * binary128 ("quad", unit roundoff 2^-113, Table 1 of the paper):
 *
 *  - oracle_eigvals: classical Sturm-sequence bisection on T itself (the
 *    bisection the paper refers to for eigenvalue approximation, Sec. 2,
 *    "Classification of the eigenvalues").  It never forms an LDL^T
 *    representation, never shifts and never perturbs.
 *  - oracle_eigvecs: inverse iteration with the quad eigenvalue as shift,
 *    tridiagonal Gaussian elimination with partial pivoting, and modified
 *    Gram-Schmidt against the already accepted vectors of nearby eigenvalues.
 *  - oracle_jacobi: cyclic Jacobi on a dense symmetric matrix (brute force,
 *    used only to pin the two routines above on tiny inputs).
 *  - oracle_residual_ortho: the accuracy measures R and O of Eq. (1.1)
 *    (label def:defresortho), accumulated in quad.
 *
 * The quad type is __float128 on x86-64 and `long double` on AArch64 Linux,
 * where that type is IEEE binary128.  No quad math library is needed: the
 * only transcendental operation, the square root, is a Newton iteration
 * seeded from the double-precision root.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#if defined(__aarch64__)
typedef long double qreal;
_Static_assert(LDBL_MANT_DIG == 113, "long double must be IEEE binary128 on this target");
#else
typedef __float128 qreal;
#endif

/* unit roundoff of binary128, Table 1 */
#define EPS_Q ((qreal)1.0 / ((qreal)(1ULL << 56) * (qreal)(1ULL << 57)))

static qreal qabs(qreal x) { return x < 0 ? -x : x; }
static qreal qmax(qreal a, qreal b) { return a > b ? a : b; }

/* Square root by Newton's method x <- (x + a/x)/2 from the double root;
 * two steps take 53 correct bits to well over 113. */
static qreal qsqrt(qreal a) {
    if (a <= 0) return 0;
    qreal x = (qreal)sqrt((double)a);
    if (x == 0) x = a; /* below the double range: start from a (converges, slowly) */
    for (int it = 0; it < 200; it++) {
        qreal nx = (x + a / x) / 2;
        if (nx == x) break;
        x = nx;
    }
    return x;
}

static int nthreads_or_default(int nthreads) {
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

int oracle_max_threads(void) { return nthreads_or_default(0); }

/* ||T||_1 = max column sum of |T| (= max row sum for symmetric T). */
static qreal tnorm1(int n, const double *d, const double *e) {
    qreal m = 0;
    for (int i = 0; i < n; i++) {
        qreal s = qabs((qreal)d[i]);
        if (i > 0) s += qabs((qreal)e[i - 1]);
        if (i < n - 1) s += qabs((qreal)e[i]);
        m = qmax(m, s);
    }
    return m;
}

/* Sturm count: number of eigenvalues of T strictly below x.
 * q_1 = d_1 - x, q_i = (d_i - x) - e_{i-1}^2 / q_{i-1}; count the q_i < 0.
 * A pivot with |q_i| <= pivmin is replaced by -pivmin (counted negative). */
static int sturm_count(int n, const double *d, const qreal *e2, qreal x, qreal pivmin) {
    int cnt = 0;
    qreal q = (qreal)d[0] - x;
    if (qabs(q) <= pivmin) q = -pivmin;
    if (q < 0) cnt++;
    for (int i = 1; i < n; i++) {
        q = ((qreal)d[i] - x) - e2[i - 1] / q;
        if (qabs(q) <= pivmin) q = -pivmin;
        if (q < 0) cnt++;
    }
    return cnt;
}

/*
 * Eigenvalues il..iu (1-based, inclusive; lambda_1 <= ... <= lambda_n) of
 * the tridiagonal T with diagonal d[0..n-1] and off-diagonal e[0..n-2].
 * Each eigenvalue is bisected independently from the Gershgorin interval
 * until hi - lo <= max(4 eps_q max(|lo|,|hi|), eps_q ||T||_1); the midpoint is
 * returned as the unevaluated sum w_hi[j] + w_lo[j] of two doubles.
 * Returns 0, or -1 on bad arguments / non-finite input.
 */
int oracle_eigvals(int n, const double *d, const double *e, int il, int iu,
                   double *w_hi, double *w_lo, int nthreads) {
    if (n < 1 || il < 1 || iu > n || il > iu) return -1;
    for (int i = 0; i < n; i++) if (!isfinite(d[i])) return -1;
    for (int i = 0; i < n - 1; i++) if (!isfinite(e[i])) return -1;
    qreal *e2 = (qreal *)malloc(sizeof(qreal) * (size_t)(n > 1 ? n - 1 : 1));
    qreal maxe2 = 1;
    for (int i = 0; i < n - 1; i++) {
        e2[i] = (qreal)e[i] * (qreal)e[i];
        maxe2 = qmax(maxe2, e2[i]);
    }
    qreal pivmin = maxe2 * EPS_Q * EPS_Q; /* far below any pivot that matters */
    qreal gl = 0, gu = 0;
    for (int i = 0; i < n; i++) {
        qreal r = 0;
        if (i > 0) r += qabs((qreal)e[i - 1]);
        if (i < n - 1) r += qabs((qreal)e[i]);
        qreal lo = (qreal)d[i] - r, hi = (qreal)d[i] + r;
        if (i == 0 || lo < gl) gl = lo;
        if (i == 0 || hi > gu) gu = hi;
    }
    qreal tn = tnorm1(n, d, e);
    qreal pad = 2 * EPS_Q * tn * n + pivmin;
    gl -= pad;
    gu += pad;
    qreal tolabs = EPS_Q * (tn > 0 ? tn : 1);
    int nt = nthreads_or_default(nthreads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int j = il; j <= iu; j++) {
        qreal lo = gl, hi = gu; /* invariant: count(lo) < j <= count(hi) */
        for (int it = 0; it < 400; it++) {
            qreal width = hi - lo;
            qreal tol = qmax(4 * EPS_Q * qmax(qabs(lo), qabs(hi)), tolabs);
            if (width <= tol) break;
            qreal mid = lo + width / 2;
            if (mid <= lo || mid >= hi) break;
            if (sturm_count(n, d, e2, mid, pivmin) >= j) hi = mid;
            else lo = mid;
        }
        qreal m = lo + (hi - lo) / 2;
        double h = (double)m;
        w_hi[j - il] = h;
        w_lo[j - il] = (double)(m - (qreal)h);
    }
    free(e2);
    return 0;
}

/* Sturm count of T at x (number of eigenvalues below x), exposed for tests. */
int oracle_sturm_count(int n, const double *d, const double *e, double x_hi, double x_lo) {
    if (n < 1) return -1;
    qreal *e2 = (qreal *)malloc(sizeof(qreal) * (size_t)(n > 1 ? n - 1 : 1));
    qreal maxe2 = 1;
    for (int i = 0; i < n - 1; i++) {
        e2[i] = (qreal)e[i] * (qreal)e[i];
        maxe2 = qmax(maxe2, e2[i]);
    }
    int c = sturm_count(n, d, e2, (qreal)x_hi + (qreal)x_lo, maxe2 * EPS_Q * EPS_Q);
    free(e2);
    return c;
}

/* SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): start vectors for inverse iteration only. */
static uint64_t splitmix64(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/*
 * Solve (T - lam I) y = b with Gaussian elimination and partial pivoting
 * (row interchanges between neighbouring rows).  The factor is upper
 * triangular with two super-diagonals.  A zero pivot is replaced by tiny.
 * Work arrays: dd, du, du2 of length n; y holds b on entry, the solution on
 * exit.
 */
static void tri_solve_pivot(int n, const double *d, const double *e, qreal lam, qreal tiny,
                            qreal *dg, qreal *du, qreal *du2, qreal *dl, int *swp, qreal *y) {
    /* rows: sub-diagonal dl[i] = e[i] (row i+1, col i), diagonal dg, super du */
    for (int i = 0; i < n; i++) {
        dg[i] = (qreal)d[i] - lam;
        du[i] = (i < n - 1) ? (qreal)e[i] : 0;
        du2[i] = 0;
        dl[i] = (i < n - 1) ? (qreal)e[i] : 0;
        swp[i] = 0;
    }
    for (int i = 0; i < n - 1; i++) {
        if (qabs(dg[i]) >= qabs(dl[i])) {
            /* no interchange: eliminate dl[i] with row i */
            if (dg[i] == 0) dg[i] = tiny;
            qreal m = dl[i] / dg[i];
            dl[i] = m;
            dg[i + 1] -= m * du[i];
            /* du2[i] stays 0 */
        } else {
            /* interchange rows i and i+1 */
            swp[i] = 1;
            qreal m = dg[i] / dl[i];
            dg[i] = dl[i];
            dl[i] = m;
            qreal t = du[i];
            du[i] = dg[i + 1];
            dg[i + 1] = t - m * dg[i + 1];
            if (i < n - 2) {
                du2[i] = du[i + 1];
                du[i + 1] = -m * du[i + 1];
            }
        }
    }
    if (dg[n - 1] == 0) dg[n - 1] = tiny;
    /* forward: apply the row operations to y */
    for (int i = 0; i < n - 1; i++) {
        if (swp[i]) {
            qreal t = y[i];
            y[i] = y[i + 1];
            y[i + 1] = t - dl[i] * y[i + 1];
        } else {
            y[i + 1] -= dl[i] * y[i];
        }
    }
    /* back substitution with U (diag dg, super du, super-super du2) */
    y[n - 1] /= dg[n - 1];
    if (n > 1) y[n - 2] = (y[n - 2] - du[n - 2] * y[n - 1]) / dg[n - 2];
    for (int i = n - 3; i >= 0; i--)
        y[i] = (y[i] - du[i] * y[i + 1] - du2[i] * y[i + 2]) / dg[i];
}

/*
 * Eigenvectors by inverse iteration in quad for the k eigenvalues
 * lam[j] = lam_hi[j] + lam_lo[j] (ascending).  Vector j starts from a
 * seeded random vector, and each of `iters` steps solves (T - lam_j I) y = x,
 * orthogonalises y (modified Gram-Schmidt, twice) against every accepted
 * vector i < j with |lam_i - lam_j| <= gs_window * ||T||_1, and normalises.
 * The sign is fixed so that the entry of largest magnitude (first one on
 * ties) is positive.  Z is column-major with leading dimension ldz (double).
 * Returns 0, or -1 on bad arguments.
 */
int oracle_eigvecs(int n, const double *d, const double *e, int k, const double *lam_hi,
                   const double *lam_lo, double *Z, int ldz, double gs_window, int iters,
                   uint64_t seed) {
    if (n < 1 || k < 0 || k > n || ldz < n || iters < 1) return -1;
    qreal tn = tnorm1(n, d, e);
    if (tn == 0) tn = 1;
    qreal tiny = EPS_Q * tn;
    qreal win = (qreal)gs_window * tn;
    size_t nn = (size_t)n;
    qreal *V = (qreal *)malloc(sizeof(qreal) * nn * (size_t)(k > 0 ? k : 1)); /* accepted vectors */
    qreal *w = (qreal *)malloc(sizeof(qreal) * nn * 5);
    int *swp = (int *)malloc(sizeof(int) * nn);
    qreal *y = (qreal *)malloc(sizeof(qreal) * nn);
    qreal *lam = (qreal *)malloc(sizeof(qreal) * (size_t)(k > 0 ? k : 1));
    for (int j = 0; j < k; j++) lam[j] = (qreal)lam_hi[j] + (qreal)lam_lo[j];
    uint64_t st = seed;
    for (int j = 0; j < k; j++) {
        qreal *x = V + (size_t)j * nn;
        for (int i = 0; i < n; i++) {
            uint64_t r = splitmix64(&st);
            x[i] = (qreal)((double)(r >> 11) * (1.0 / 9007199254740992.0)) * 2 - 1;
        }
        int jlo = j;
        while (jlo > 0 && qabs(lam[j] - lam[jlo - 1]) <= win) jlo--;
        for (int it = 0; it < iters; it++) {
            memcpy(y, x, sizeof(qreal) * nn);
            tri_solve_pivot(n, d, e, lam[j], tiny, w, w + nn, w + 2 * nn, w + 3 * nn, swp, y);
            for (int pass = 0; pass < 2; pass++) {
                for (int i = jlo; i < j; i++) {
                    const qreal *v = V + (size_t)i * nn;
                    qreal dot = 0;
                    for (int r = 0; r < n; r++) dot += v[r] * y[r];
                    for (int r = 0; r < n; r++) y[r] -= dot * v[r];
                }
            }
            qreal s = 0;
            for (int r = 0; r < n; r++) s += y[r] * y[r];
            s = qsqrt(s);
            if (s == 0) { /* degenerate: restart from a unit vector */
                for (int r = 0; r < n; r++) y[r] = 0;
                y[j % n] = 1;
                s = 1;
            }
            for (int r = 0; r < n; r++) x[r] = y[r] / s;
        }
        int imax = 0;
        for (int r = 1; r < n; r++) if (qabs(x[r]) > qabs(x[imax])) imax = r;
        if (x[imax] < 0) for (int r = 0; r < n; r++) x[r] = -x[r];
        for (int r = 0; r < n; r++) Z[(size_t)j * (size_t)ldz + r] = (double)x[r];
    }
    free(V); free(w); free(swp); free(y); free(lam);
    return 0;
}

/*
 * Cyclic Jacobi for a dense symmetric n x n matrix A (column-major, double
 * input), in quad.  Returns the eigenvalues ascending in w_hi + w_lo and, if
 * V != NULL, the eigenvectors (column-major, ldv = n, largest entry made
 * positive).  Sweeps until every off-diagonal entry is below eps_q times the
 * Frobenius norm.  Intended for n <= 64.  Returns the sweep count or -1.
 */
int oracle_jacobi(int n, const double *A, double *w_hi, double *w_lo, double *V) {
    if (n < 1 || n > 512) return -1;
    size_t nn = (size_t)n;
    qreal *a = (qreal *)malloc(sizeof(qreal) * nn * nn);
    qreal *v = (qreal *)malloc(sizeof(qreal) * nn * nn);
    for (size_t i = 0; i < nn * nn; i++) a[i] = (qreal)A[i];
    for (size_t i = 0; i < nn; i++)
        for (size_t j = 0; j < nn; j++) v[i + j * nn] = (i == j) ? 1 : 0;
    qreal fro = 0;
    for (size_t i = 0; i < nn * nn; i++) fro += a[i] * a[i];
    fro = qsqrt(fro);
    int sweep;
    for (sweep = 0; sweep < 100; sweep++) {
        qreal off = 0;
        for (int p = 0; p < n; p++)
            for (int q = p + 1; q < n; q++) off = qmax(off, qabs(a[p + q * nn]));
        if (off <= EPS_Q * EPS_Q * fro || off == 0) break;
        for (int p = 0; p < n - 1; p++) {
            for (int q = p + 1; q < n; q++) {
                qreal apq = a[p + q * nn];
                if (apq == 0) continue;
                qreal app = a[p + p * nn], aqq = a[q + q * nn];
                /* rotation angle from zeta = (a_qq - a_pp) / (2 a_pq) */
                qreal zeta = (aqq - app) / (2 * apq);
                qreal t = 1 / (qabs(zeta) + qsqrt(1 + zeta * zeta));
                if (zeta < 0) t = -t;
                qreal c = 1 / qsqrt(1 + t * t), s = c * t;
                for (int r = 0; r < n; r++) { /* columns p, q: A <- A J */
                    qreal arp = a[r + p * nn], arq = a[r + q * nn];
                    a[r + p * nn] = c * arp - s * arq;
                    a[r + q * nn] = s * arp + c * arq;
                }
                for (int r = 0; r < n; r++) { /* rows p, q: A <- J^T A */
                    qreal apr = a[p + r * nn], aqr = a[q + r * nn];
                    a[p + r * nn] = c * apr - s * aqr;
                    a[q + r * nn] = s * apr + c * aqr;
                }
                a[p + q * nn] = 0;
                a[q + p * nn] = 0;
                for (int r = 0; r < n; r++) {
                    qreal vrp = v[r + p * nn], vrq = v[r + q * nn];
                    v[r + p * nn] = c * vrp - s * vrq;
                    v[r + q * nn] = s * vrp + c * vrq;
                }
            }
        }
    }
    /* selection sort of the eigenvalues, carrying the vectors */
    int *idx = (int *)malloc(sizeof(int) * nn);
    for (int i = 0; i < n; i++) idx[i] = i;
    for (int i = 0; i < n; i++) {
        int m = i;
        for (int j = i + 1; j < n; j++)
            if (a[idx[j] + idx[j] * nn] < a[idx[m] + idx[m] * nn]) m = j;
        int t = idx[i]; idx[i] = idx[m]; idx[m] = t;
    }
    for (int i = 0; i < n; i++) {
        qreal lamq = a[idx[i] + idx[i] * nn];
        double h = (double)lamq;
        w_hi[i] = h;
        w_lo[i] = (double)(lamq - (qreal)h);
        if (V) {
            const qreal *col = v + (size_t)idx[i] * nn;
            int imax = 0;
            for (int r = 1; r < n; r++) if (qabs(col[r]) > qabs(col[imax])) imax = r;
            qreal sg = col[imax] < 0 ? -1 : 1;
            for (int r = 0; r < n; r++) V[(size_t)i * nn + r] = (double)(sg * col[r]);
        }
    }
    free(idx); free(a); free(v);
    return sweep;
}

/*
 * Accuracy measures of Eq. (1.1): for k computed pairs (W[j], Z[:, j])
 * of T (Z column-major, leading dimension ldz, double), returns
 *   res[j]  = ||T z_j - W_j z_j||_1 / ||T||_1           (R = max_j res[j])
 *   res2[j] = ||T z_j - W_j z_j||_2                      (absolute 2-norm)
 *   *ortho  = max_{i != j} |z_i^T z_j|                   (O)
 *   *ortho_diag = max_j |z_j^T z_j - 1|
 * all accumulated in quad.  Cost O(n k^2): meant for n, k up to ~1000.
 */
int oracle_residual_ortho(int n, const double *d, const double *e, int k, const double *W,
                          const double *Z, int ldz, double *res, double *res2, double *ortho,
                          double *ortho_diag, int nthreads) {
    if (n < 1 || k < 0 || ldz < n) return -1;
    qreal tn = tnorm1(n, d, e);
    if (tn == 0) tn = 1;
    int nt = nthreads_or_default(nthreads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
    for (int j = 0; j < k; j++) {
        const double *z = Z + (size_t)j * (size_t)ldz;
        qreal lam = (qreal)W[j], s1 = 0, s2 = 0;
        for (int i = 0; i < n; i++) {
            qreal r = ((qreal)d[i] - lam) * (qreal)z[i];
            if (i > 0) r += (qreal)e[i - 1] * (qreal)z[i - 1];
            if (i < n - 1) r += (qreal)e[i] * (qreal)z[i + 1];
            s1 += qabs(r);
            s2 += r * r;
        }
        res[j] = (double)(s1 / tn);
        res2[j] = (double)qsqrt(s2);
    }
    qreal omax = 0, dmax = 0;
#pragma omp parallel num_threads(nt)
    {
        qreal lo = 0, ld = 0;
#pragma omp for schedule(dynamic, 4)
        for (int j = 0; j < k; j++) {
            const double *zj = Z + (size_t)j * (size_t)ldz;
            for (int i = 0; i <= j; i++) {
                const double *zi = Z + (size_t)i * (size_t)ldz;
                qreal s = 0;
                for (int r = 0; r < n; r++) s += (qreal)zi[r] * (qreal)zj[r];
                if (i == j) ld = qmax(ld, qabs(s - 1));
                else lo = qmax(lo, qabs(s));
            }
        }
#pragma omp critical
        {
            omax = qmax(omax, lo);
            dmax = qmax(dmax, ld);
        }
    }
    *ortho = (double)omax;
    *ortho_diag = (double)dmax;
    return 0;
}
