"""Pins for the oracle (CPU only): closed forms, brute force, invariants and
library routines -- each chosen so that a plausible slip in the oracle (a
dropped term, a wrong sign or index, a missing Gram-Schmidt step) fails one.
"""
import os
import re
import shutil
import subprocess
import tempfile

import mpmath
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from oracle import metrics
from paper_1304_1864_gb300 import inputs

mpmath.mp.dps = 50
EPS_Q = 2.0 ** -113
EPS_D = 2.0 ** -53
# the oracle returns binary128 values as hi + lo doubles (106 bits): compare at 2^-100
TOL_HL = 2.0 ** -100


def _mp(hi, lo):
    return mpmath.mpf(float(hi)) + mpmath.mpf(float(lo))


@pytest.mark.parametrize("n", [1, 2, 3, 10, 257])
def test_121_eigenvalues_closed_form(n):
    # 1-2-1: lambda_k = 2 - 2 cos(k pi / (n+1)), exact input -> quad accuracy
    d, e = inputs.one_two_one(n)
    hi, lo = oracle.eigvals(d, e)
    for k in range(1, n + 1):
        exact = 2 - 2 * mpmath.cos(k * mpmath.pi / (n + 1))
        assert abs(_mp(hi[k - 1], lo[k - 1]) - exact) <= TOL_HL * 4


def test_121_eigenvalue_subset_indices():
    n = 64
    d, e = inputs.one_two_one(n)
    hi, lo = oracle.eigvals(d, e, il=17, iu=20)
    for j, k in enumerate(range(17, 21)):
        exact = 2 - 2 * mpmath.cos(k * mpmath.pi / (n + 1))
        assert abs(_mp(hi[j], lo[j]) - exact) <= TOL_HL * 4


@pytest.mark.parametrize("n", [1, 2, 9, 100])
def test_121_eigenvectors_closed_form(n):
    # z_k[i] = sqrt(2/(n+1)) sin(i k pi/(n+1)), sign: largest entry positive
    d, e = inputs.one_two_one(n)
    hi, lo = oracle.eigvals(d, e)
    Z = oracle.eigvecs(d, e, hi, lo)
    i = np.arange(1, n + 1)[:, None]
    k = np.arange(1, n + 1)[None, :]
    Zx = np.sqrt(2.0 / (n + 1)) * np.sin(i * k * np.pi / (n + 1))
    # eigenvectors are unique up to sign only (ties in the largest entry make
    # the sign convention rounding-dependent), so compare sign-free
    assert np.max(metrics.sin_angles(Z, Zx)) <= 1e-13
    # the sign convention: an entry of largest magnitude is positive (up to
    # rounding on ties)
    assert np.all(Z.max(axis=0) >= np.abs(Z).max(axis=0) * (1 - 1e-13))


@pytest.mark.parametrize("n", [2, 51, 400])
def test_clement_integer_spectrum(n):
    # eigenvalues -(n-1), -(n-3), ..., n-1; the double rounding of e_i =
    # sqrt(i(n-i)) moves them by at most ||dT||_2 <= 2 max|de_i| <= 2 eps_d max e_i
    d, e = inputs.clement(n)
    hi, lo = oracle.eigvals(d, e)
    exact = np.arange(-(n - 1), n, 2, dtype=np.float64)
    err = np.abs((hi - exact) + lo)
    assert np.max(err) <= 2 * EPS_D * np.max(e) * 1.01 + 1e-30


def test_sturm_count_brackets_each_eigenvalue():
    d, e = inputs.uniform_random(60, 7)
    hi, lo = oracle.eigvals(d, e)
    for j in range(60):
        lam = hi[j]
        delta = 1e-9
        assert oracle.sturm_count(d, e, lam - delta) == j
        assert oracle.sturm_count(d, e, lam + delta) == j + 1
    assert oracle.sturm_count(d, e, -10.0) == 0
    assert oracle.sturm_count(d, e, 10.0) == 60


@pytest.mark.parametrize("case", ["rand1", "rand2", "rand5", "rand17", "rand64", "wilk21", "glued3x7", "zeros"])
def test_bisection_and_inverse_iteration_match_dense_jacobi(case):
    if case.startswith("rand"):
        n = int(case[4:])
        d, e = inputs.uniform_random(n, n)
    elif case == "wilk21":
        d, e = inputs.wilkinson(21)
    elif case == "glued3x7":
        d, e = inputs.glued_wilkinson(3, 7, 1e-3)
    else:
        d, e = np.zeros(6), np.zeros(5)
    n = d.size
    A = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    jh, jl, V = oracle.jacobi(A)
    hi, lo = oracle.eigvals(d, e)
    tn = max(metrics.tnorm1(d, e), 1.0)
    assert np.max(np.abs((jh - hi) + (jl - lo))) <= 1e-28 * tn
    if case == "zeros":
        return
    Z = oracle.eigvecs(d, e, hi, lo)
    lam = hi + lo
    gaps = np.full(n, np.inf)
    if n > 1:
        g = np.diff(lam)
        gaps[:-1] = np.minimum(gaps[:-1], g)
        gaps[1:] = np.minimum(gaps[1:], g)
    sep = gaps > 1e-6 * tn
    assert np.all(metrics.sin_angles(Z[:, sep], V[:, sep]) <= 1e-14)


def test_jacobi_pinned_to_lapack():
    # the brute-force pin itself agrees with LAPACK's dense solver
    rng = np.random.default_rng(11)
    A = rng.standard_normal((24, 24))
    A = A + A.T
    jh, jl, V = oracle.jacobi(A)
    w, U = np.linalg.eigh(A)
    assert np.max(np.abs(jh - w)) <= 1e-13 * np.max(np.abs(w))
    assert np.max(metrics.sin_angles(V, U)) <= 1e-12


@pytest.mark.parametrize("kind,n", [("uniform", 300), ("glued", 210), ("wilkinson", 201), ("hermite", 150)])
def test_eigenvalues_match_lapack_tridiagonal(kind, n):
    d, e = inputs.make(kind, n, seed=3)
    hi, lo = oracle.eigvals(d, e)
    w = sla.eigh_tridiagonal(d, e, eigvals_only=True)
    tn = metrics.tnorm1(d, e)
    assert np.max(np.abs(hi - w)) <= 50 * d.size * EPS_D * tn


@pytest.mark.parametrize("kind,n", [("uniform", 200), ("wilkinson", 41), ("clement", 64)])
def test_trace_and_frobenius_invariants(kind, n):
    # sum(lambda) = trace T, sum(lambda^2) = ||T||_F^2
    d, e = inputs.make(kind, n, seed=5)
    hi, lo = oracle.eigvals(d, e)
    lam = [_mp(h, l) for h, l in zip(hi, lo)]
    tr = mpmath.fsum(mpmath.mpf(float(x)) for x in d)
    fro = mpmath.fsum(mpmath.mpf(float(x)) ** 2 for x in d) + 2 * mpmath.fsum(mpmath.mpf(float(x)) ** 2 for x in e)
    scale = max(1.0, metrics.tnorm1(d, e))
    assert abs(mpmath.fsum(lam) - tr) <= 1e-28 * scale * n
    assert abs(mpmath.fsum(x * x for x in lam) - fro) <= 1e-28 * scale ** 2 * n


def test_hermite_roots():
    n = 40
    d, e = inputs.hermite(n)
    hi, lo = oracle.eigvals(d, e)
    roots = np.polynomial.hermite.hermgauss(n)[0]
    assert np.max(np.abs(hi - np.sort(roots))) <= 1e-12


def test_inverse_iteration_orthogonal_on_exact_ties():
    # two identical decoupled blocks: every eigenvalue is exactly double, so
    # only the Gram-Schmidt step can make the two vectors orthogonal
    db, eb = inputs.wilkinson(11)
    d = np.concatenate([db, db])
    e = np.concatenate([eb, [0.0], eb])
    hi, lo = oracle.eigvals(d, e)
    Z = oracle.eigvecs(d, e, hi, lo)
    m = oracle.residual_ortho(d, e, hi + lo, Z)
    assert m["O"] <= 4 * EPS_D
    assert m["O_diag"] <= 4 * EPS_D
    assert m["R"] <= 4 * EPS_D


def test_residual_ortho_measures_known_error():
    # planted error: rotate two eigenvectors by a known angle -> O = sin cos
    d, e = inputs.one_two_one(30)
    hi, lo = oracle.eigvals(d, e)
    Z = oracle.eigvecs(d, e, hi, lo)
    th = 1e-7
    Zp = Z.copy()
    Zp[:, 3] = np.cos(th) * Z[:, 3] + np.sin(th) * Z[:, 4]
    m = oracle.residual_ortho(d, e, hi, Zp)
    assert abs(m["O"] - np.sin(th) * np.cos(th)) <= 1e-15
    # residual of the rotated vector: sin(th) |lambda_4 - lambda_3| in 2-norm
    assert abs(m["res2"][3] - np.sin(th) * (hi[4] - hi[3])) <= 1e-15


def test_large_n_metrics_agree_with_quad():
    d, e = inputs.uniform_random(180, 9)
    hi, lo = oracle.eigvals(d, e)
    Z = oracle.eigvecs(d, e, hi, lo)
    rng = np.random.default_rng(1)
    Zp = Z + 1e-12 * rng.standard_normal(Z.shape)
    q = oracle.residual_ortho(d, e, hi, Zp)
    r2, r1 = metrics.residuals(d, e, hi, Zp)
    assert np.allclose(r2, q["res2"], rtol=1e-6, atol=1e-30)
    off, dia = metrics.ortho(Zp, target=1e-12)
    assert abs(off - q["O"]) <= 1e-3 * q["O"]
    assert abs(dia - q["O_diag"]) <= 1e-3 * q["O_diag"]


def test_dd_helpers_exact():
    from fractions import Fraction
    rng = np.random.default_rng(2)
    a = rng.standard_normal(200) * 10.0 ** rng.integers(-20, 20, 200)
    b = rng.standard_normal(200) * 10.0 ** rng.integers(-20, 20, 200)
    p, q = metrics.two_prod(a, b)
    s, t = metrics.two_sum(a, b)
    for i in range(200):
        assert Fraction(p[i]) + Fraction(q[i]) == Fraction(a[i]) * Fraction(b[i])
        assert Fraction(s[i]) + Fraction(t[i]) == Fraction(a[i]) + Fraction(b[i])


# --------------------------------------------------- mutants must fail a pin

MUTANTS = {
    # wrong sign of the off-diagonal term in the Sturm recurrence
    "sturm_sign": (r"q = \(\(qreal\)d\[i\] - x\) - e2\[i - 1\] / q;", "q = ((qreal)d[i] - x) + e2[i - 1] / q;"),
    # off-by-one in the eigenvalue index
    "index": (r"if \(sturm_count\(n, d, e2, mid, pivmin\) >= j\) hi = mid;",
              "if (sturm_count(n, d, e2, mid, pivmin) >= j + 1) hi = mid;"),
    # Gram-Schmidt dropped
    "no_gs": (r"while \(jlo > 0 && qabs\(lam\[j\] - lam\[jlo - 1\]\) <= win\) jlo--;", ""),
    # fill-in of the pivoted elimination dropped from the back substitution
    "no_fill": (r"y\[i\] = \(y\[i\] - du\[i\] \* y\[i \+ 1\] - du2\[i\] \* y\[i \+ 2\]\) / dg\[i\];",
                "y[i] = (y[i] - du[i] * y[i + 1]) / dg[i];"),
}


def _build_mutant(tmp, name):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    pat, rep = MUTANTS[name]
    mutated, cnt = re.subn(pat, rep, src)
    assert cnt == 1, name
    c = os.path.join(tmp, "m.c")
    so = os.path.join(tmp, "libm_%s.so" % name)
    open(c, "w").write(mutated)
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-fopenmp", "-std=gnu11", c, "-o", so, "-lm"], check=True)
    return so


def _pins_pass(so):
    """Run a subset of the pins against a library built from `so`."""
    import oracle as om
    saved = om._lib
    try:
        om._lib = None
        orig = om._build.build
        om._build.build = lambda force=False: so
        try:
            om.lib()
        finally:
            om._build.build = orig
        ok = True
        try:
            test_121_eigenvalues_closed_form(10)
            test_121_eigenvectors_closed_form(9)
            test_inverse_iteration_orthogonal_on_exact_ties()
        except AssertionError:
            ok = False
        return ok
    finally:
        om._lib = saved


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistakes_fail_the_pins(name):
    tmp = tempfile.mkdtemp()
    try:
        so = _build_mutant(tmp, name)
        assert not _pins_pass(so), "mutant %s survived the pins" % name
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
