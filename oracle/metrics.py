"""Accuracy measures for large n -- TEST INFRASTRUCTURE ONLY (see oracle/__init__).

The paper measures a computed eigen-decomposition by the largest residual
norm R and the orthogonality O of Eq. (1.1) (label def:defresortho):

    R = max_i ||T z_i - lambda_i z_i||_1 / ||T||_1,
    O = max_{i != j} |z_j^T z_i|.

A plain double-precision Z^T Z carries an error of order n*eps_d itself and
cannot certify an n*eps_d target, so these routines accumulate exactly where
it matters:

* residuals: every product e_i z_j and (d_i - lambda) z_i is formed exactly as
  a double-double (Dekker split / Knuth two-sum), so the residual is exact to
  a few units of 2^-104 relative to ||T||;
* Z^T Z: rows are taken in blocks of ``b``; each block product is one float64
  GEMM whose rounding error is at most b*eps_d*||z_i|| ||z_j|| (any summation
  order), and the block results are summed in double-double.  ``b`` is chosen
  so that b*eps_d is at most ``slack`` times the caller's target.
"""
import numpy as np

EPS_D = 2.0 ** -53
EPS_S = 2.0 ** -24
_SPLIT = 134217729.0  # 2^27 + 1 (Dekker's splitting constant for binary64)


def two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def _split(a):
    c = _SPLIT * a
    hi = c - (c - a)
    return hi, a - hi


def two_prod(a, b):
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    return p, ((ah * bh - p) + ah * bl + al * bh) + al * bl


def dd_add(ah, al, bh, bl):
    s, t = two_sum(ah, bh)
    t = t + al + bl
    return two_sum(s, t)


def tnorm1(d, e):
    d = np.abs(np.asarray(d, dtype=np.float64))
    e = np.abs(np.asarray(e, dtype=np.float64))
    s = d.copy()
    if e.size:
        s[:-1] += e
        s[1:] += e
    return float(s.max()) if s.size else 0.0


def residuals(d, e, W, Z, panel=256):
    """Per-column exact-ish residual 2-norms and 1-norms ||T z_j - W_j z_j||."""
    d = np.asarray(d, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    n, k = Z.shape
    r2 = np.empty(k)
    r1 = np.empty(k)
    for c0 in range(0, k, panel):
        c1 = min(k, c0 + panel)
        z = np.asarray(Z[:, c0:c1], dtype=np.float64)
        lam = W[c0:c1][None, :]
        # (d_i - lambda) as a double-double, times z_i exactly
        sh, sl = two_sum(d[:, None], -lam)
        ph, pl = two_prod(sh, z)
        pl = pl + sl * z
        if n > 1:
            # + e_{i-1} z_{i-1}
            qh, ql = two_prod(e[:, None], z[:-1, :])
            h, l = dd_add(ph[1:, :], pl[1:, :], qh, ql)
            ph = ph.copy()
            pl = pl.copy()
            ph[1:, :], pl[1:, :] = h, l
            # + e_i z_{i+1}
            qh, ql = two_prod(e[:, None], z[1:, :])
            h, l = dd_add(ph[:-1, :], pl[:-1, :], qh, ql)
            ph[:-1, :], pl[:-1, :] = h, l
        r = ph + pl
        r2[c0:c1] = np.sqrt(np.sum(r * r, axis=0))
        r1[c0:c1] = np.sum(np.abs(r), axis=0)
    return r2, r1


def ortho(Z, target, slack=0.05, panel=1024):
    """Return (max_{i!=j} |z_i^T z_j|, max_j |z_j^T z_j - 1|) for the columns of
    Z, with accumulation error at most about ``slack * target``."""
    Z = np.asarray(Z)
    n, k = Z.shape
    b = int(max(8, min(n, slack * target / EPS_D)))
    Zd = np.asarray(Z, dtype=np.float64)
    off = 0.0
    dia = 0.0
    for c0 in range(0, k, panel):
        c1 = min(k, c0 + panel)
        sh = np.zeros((k, c1 - c0))
        sl = np.zeros((k, c1 - c0))
        for r0 in range(0, n, b):
            r1 = min(n, r0 + b)
            blk = Zd[r0:r1, :].T @ Zd[r0:r1, c0:c1]
            sh, t = two_sum(sh, blk)
            sl = sl + t
        g = sh + sl  # Z^T Z[:, c0:c1] (rows: all columns of Z)
        idx = np.arange(c0, c1)
        diag = g[idx, idx - c0].copy()
        dia = max(dia, float(np.max(np.abs(diag - 1.0))))
        g[idx, idx - c0] = 0.0
        off = max(off, float(np.max(np.abs(g))))
    return off, dia


def sin_angles(U, V):
    """Sine of the angle between matching unit columns of U and V (sign-free),
    computed as min(||u - v||, ||u + v||) * sqrt(1 - ||u-v||^2/4) -- exact for
    unit vectors and accurate for tiny angles."""
    U = np.asarray(U, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    dm = np.linalg.norm(U - V, axis=0)
    dp = np.linalg.norm(U + V, axis=0)
    m = np.minimum(dm, dp)
    return m * np.sqrt(np.maximum(0.0, 1.0 - m * m / 4.0))


def subspace_sin(U, V):
    """Sine of the largest principal angle between span(U) and span(V)
    (both with orthonormal columns): ||U - V (V^T U)||_2."""
    U = np.asarray(U, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    R = U - V @ (V.T @ U)
    return float(np.linalg.norm(R, 2)) if R.size else 0.0
