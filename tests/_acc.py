"""Shared accuracy checks for the GPU parity tests (compare against the oracle)."""
import numpy as np

import oracle
from oracle import metrics

EPS = {"s": 2.0 ** -24, "d": 2.0 ** -53}

# Tolerances (in units of n eps_x ||T||_1 for residuals and eigenvalues,
# n eps_x for orthogonality).  Mixed precision: the targets the method is
# meant to reach (eigenvalues within 2 n eps ||T||, residual and
# orthogonality <= 1).  Plain (y = x): Eq. (2.2) stops the RQI at
# k_rs gap n eps / gaptol and Theorem 1 bounds orthogonality by
# O(n eps / gaptol); with gaptol = 1e-3 (x = d) or 3e-3 (x = s) that is
# 1000 n eps for both.
TOL = {
    "mixed": {"eig": 2.0, "res": 1.0, "orth": 1.0},
    "plain": {"eig": 2.0, "res": 1000.0, "orth": 1000.0},
}


def as_np(x):
    if hasattr(x, "detach"):
        return x.detach().cpu().numpy()
    return np.asarray(x)


def exact_input(d, e, prec):
    """The input exactly as the solver sees it, in float64."""
    dt = np.float32 if prec == "s" else np.float64
    return np.asarray(d, dtype=dt).astype(np.float64), np.asarray(e, dtype=dt).astype(np.float64)


def check_eigvals(d, e, W, prec, mode, idx=None, il=1):
    """Element-wise eigenvalue parity with the binary128 oracle (sampled rows
    `idx` of W if given, W[k] being eigenvalue il + k)."""
    n = d.size
    W = as_np(W).astype(np.float64)
    tn = metrics.tnorm1(d, e)
    bound = TOL[mode]["eig"] * n * EPS[prec] * tn
    if idx is None:
        idx = np.arange(W.size)
    errs = []
    for k in idx:
        j = il + int(k)
        hi, lo = oracle.eigvals(d, e, j, j)
        errs.append(abs(W[k] - (hi[0] + lo[0])))
    errs = np.array(errs)
    assert np.all(errs <= bound + 1e-300), "eigenvalue error %.3g > %.3g (max at %d)" % (
        errs.max(), bound, int(idx[int(np.argmax(errs))]))
    return errs.max() / max(bound, 1e-300)


_ORACLE_CACHE = {}


def oracle_all(name, d, e):
    """All eigenvalues (hi + lo of the binary128 bisection) of the named test
    matrix, computed once per test session (one parallel oracle sweep)."""
    if name not in _ORACLE_CACHE:
        hi, lo = oracle.eigvals(d, e)
        _ORACLE_CACHE[name] = (hi, lo)
    return _ORACLE_CACHE[name]


def check_eigvals_all(d, e, W, prec, mode, lam, il=1):
    """Every entry W[k] against the oracle eigenvalue il + k (lam = hi + lo of
    the full oracle spectrum, as two arrays), element by element, within
    2 n eps_x ||T||_1."""
    n = d.size
    W = as_np(W).astype(np.float64)
    hi, lo = lam
    ref_hi = hi[il - 1:il - 1 + W.size]
    ref_lo = lo[il - 1:il - 1 + W.size]
    # the rounding of these two subtractions is far below the bound
    err = np.abs((W - ref_hi) - ref_lo)
    bound = TOL[mode]["eig"] * n * EPS[prec] * metrics.tnorm1(d, e)
    bad = np.nonzero(~(err <= bound))[0]
    assert bad.size == 0, "%d eigenvalues off by more than %.3g (worst %.3g at %d)" % (
        bad.size, bound, err.max(), int(np.argmax(err)))
    return float(err.max() / bound)


def measure_res_orth(d, e, W, Z, prec):
    """Residual ||T z - w z||_2 / (||T||_1 n eps) and orthogonality
    max |Z^T Z - I| / (n eps), both with exact accumulation (oracle.metrics),
    without a verdict."""
    n = d.size
    W = as_np(W).astype(np.float64)
    Z = as_np(Z)
    if W.size == 0:
        return 0.0, 0.0
    tn = metrics.tnorm1(d, e)
    ne = n * EPS[prec]
    r2, _ = metrics.residuals(d, e, W, Z)
    res = float(r2.max() / (tn * ne)) if tn > 0 else float(r2.max())
    off, dia = metrics.ortho(Z, target=ne)
    return res, max(off, dia) / ne


def check_res_orth(d, e, W, Z, prec, mode):
    """measure_res_orth, asserted against the targets of the mode (TOL)."""
    res, orth = measure_res_orth(d, e, W, Z, prec)
    assert res <= TOL[mode]["res"], "residual %.3g n eps ||T|| > %.3g" % (res, TOL[mode]["res"])
    assert orth <= TOL[mode]["orth"], "orthogonality %.3g n eps > %.3g" % (orth, TOL[mode]["orth"])
    return res, orth


def check_vectors_gap_theorem(d, e, W, Z, prec, il=1, idx=None, max_n_oracle=2000):
    """Each computed vector against the oracle's (inverse iteration in
    binary128) through the Gap Theorem (Sec. 2, Eq. gapthmmain): both are
    within ||r|| / gap of the true eigenvector, so the sine of their angle is
    at most (||r_gpu|| + ||r_oracle||) / gap.  Eigenvalues whose gap is below
    1e3 n eps ||T|| are skipped (only their subspace is unique)."""
    n = d.size
    W = as_np(W).astype(np.float64)
    Z = as_np(Z).astype(np.float64)
    if idx is None:
        idx = np.arange(W.size)
    allhi, alllo = oracle.eigvals(d, e)
    lam = allhi + alllo
    tn = metrics.tnorm1(d, e)
    ne = n * EPS[prec]
    checked = 0
    for k in idx:
        j = il + int(k) - 1
        g = np.inf
        if j > 0:
            g = min(g, lam[j] - lam[j - 1])
        if j < n - 1:
            g = min(g, lam[j + 1] - lam[j])
        if g <= 1e3 * ne * tn:
            continue
        zo = oracle.eigvecs(d, e, allhi[j:j + 1], alllo[j:j + 1])[:, 0]
        z = Z[:, k]
        r_gpu = metrics.residuals(d, e, W[k:k + 1], z[:, None])[0][0]
        r_or = metrics.residuals(d, e, np.array([lam[j]]), zo[:, None])[0][0]
        s = metrics.sin_angles(z[:, None], zo[:, None])[0]
        bound = (r_gpu + r_or) / g * 1.01 + 4 * EPS[prec] * np.sqrt(n)
        assert s <= bound, "vector %d: sin angle %.3g > gap-theorem bound %.3g" % (j + 1, s, bound)
        checked += 1
    return checked


def check_sign_convention(Z, prec):
    Z = as_np(Z).astype(np.float64)
    if Z.size == 0:
        return
    amax = np.abs(Z).max(axis=0)
    assert np.all(Z.max(axis=0) >= amax * (1 - 64 * EPS[prec])), "largest entry of a column is negative"
