"""The dense symmetric eigenproblem (Sec. 5, Fig. 3): A = Q T Q^T with a random
orthogonal Q and T one of the paper's tridiagonal test types, reduced back to
tridiagonal form on the GPU, solved by the tridiagonal MRRR solver and
back-transformed (mrrr_syev_s / _d).

Checks: against the oracle's dense Jacobi (brute force, n = 48); the
eigenvalues of A against the oracle's eigenvalues of T (A is similar to T up
to the rounding of forming it); the residual ||A z - w z|| and the
orthogonality of Z in units of n eps_x; and the paper's claim that the
mixed-precision tridiagonal stage carries its accuracy over to the dense
problem (orthogonality better than with plain MRRR)."""
import numpy as np
import pytest

import oracle
from oracle import metrics
from paper_1304_1864_gb300 import inputs

from . import _acc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = {"s": 2.0 ** -24, "d": 2.0 ** -53}


def _qtq(d, e, seed):
    """A = Q T Q^T with Q the orthogonal factor of a seeded Gaussian matrix."""
    n = d.size
    rng = np.random.default_rng(seed)
    Q, R = np.linalg.qr(rng.standard_normal((n, n)))
    Q *= np.sign(np.diag(R))
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    A = Q @ T @ Q.T
    return 0.5 * (A + A.T)


def _solve(A, prec, mode, **kw):
    import paper_1304_1864_gb300 as m
    dt = torch.float32 if prec == "s" else torch.float64
    Ag = torch.tensor(A, dtype=dt, device="cuda")
    W, Z, st = m.solve_dense(Ag, mode=mode, **kw)
    torch.cuda.synchronize()
    assert st["status"] == 0, st
    return _acc.as_np(W).astype(np.float64), _acc.as_np(Z), st


def _res_orth(A, W, Z, prec):
    """max_j ||A z_j - w_j z_j||_2 / (||A||_1 n eps) and max |Z^T Z - I| / (n eps),
    with A as the solver saw it (rounded to the input precision), in binary64
    (the products of binary32 data are exact there; for binary64 data the
    evaluation error, about sqrt(n) eps_d ||A||, is far below the unit)."""
    n = A.shape[0]
    Ax = A.astype(np.float32 if prec == "s" else np.float64).astype(np.float64)
    Z64 = Z.astype(np.float64)
    R = Ax @ Z64 - Z64 * W[None, :]
    an = np.abs(Ax).sum(axis=0).max()
    ne = n * EPS[prec]
    res = np.linalg.norm(R, axis=0).max() / (an * ne)
    off, dia = metrics.ortho(Z, target=ne)
    return res, max(off, dia) / ne


@pytest.mark.parametrize("prec", ["s", "d"])
def test_dense_against_jacobi_n48(prec):
    # brute force: the oracle's dense cyclic Jacobi on the same matrix
    rng = np.random.default_rng(48)
    B = rng.uniform(-1, 1, (48, 48))
    A = (B + B.T) * 0.5
    Ax = A.astype(np.float32 if prec == "s" else np.float64).astype(np.float64)
    hi, lo, V = oracle.jacobi(Ax)
    order = np.argsort(hi + lo)
    lam = (hi + lo)[order]
    V = V[:, order]
    W, Z, st = _solve(A, prec, "mixed")
    an = np.abs(Ax).sum(axis=0).max()
    assert np.max(np.abs(W - lam)) <= 2 * 48 * EPS[prec] * an
    res, orth = _res_orth(A, W, Z, prec)
    assert res <= 1.0 and orth <= 1.0, (res, orth)
    # vectors against the oracle's through the gap theorem
    gaps = np.minimum(np.diff(lam, prepend=-np.inf), np.diff(lam, append=np.inf))
    r = np.linalg.norm(Ax @ Z.astype(np.float64) - Z.astype(np.float64) * W[None, :], axis=0)
    s = metrics.sin_angles(Z.astype(np.float64), V)
    assert np.all(s <= r / gaps * 1.01 + 8 * EPS[prec] * np.sqrt(48) + 1e-300)


DENSE_TYPES = ["uniform_spectrum", "121", "wilkinson", "clement"]


@pytest.mark.parametrize("prec", ["s", "d"])
@pytest.mark.parametrize("kind", DENSE_TYPES)
def test_dense_qtq_n500(kind, prec):
    n = 501 if kind == "wilkinson" else 500
    d, e = inputs.make(kind, n, seed=5)
    A = _qtq(d, e, seed=11)
    W, Z, st = _solve(A, prec, "mixed")
    assert W.size == n and np.all(np.diff(W) >= 0)
    # eigenvalues of A are those of T up to the rounding of forming A (and of
    # storing it in the input precision): within 2 n eps_x ||A||
    hi, lo = oracle.eigvals(d, e)
    an = np.abs(A).sum(axis=0).max()
    assert np.max(np.abs(W - (hi + lo))) <= 2 * n * EPS[prec] * an
    res, orth = _res_orth(A, W, Z, prec)
    assert res <= 1.0 and orth <= 1.0, (res, orth)
    _acc.check_sign_convention(Z, prec)


@pytest.mark.parametrize("kind", ["121", "wilkinson"])
def test_dense_mixed_orthogonality_beats_plain_fp32(kind):
    # Fig. 3: the accuracy of the mixed tridiagonal stage carries over to the
    # dense problem; plain binary32 MRRR is the comparison
    n = 1001
    d, e = inputs.make(kind, n, seed=5)
    A = _qtq(d, e, seed=12)
    Wm, Zm, _ = _solve(A, "s", "mixed")
    Wp, Zp, _ = _solve(A, "s", "plain")
    rm, om = _res_orth(A, Wm, Zm, "s")
    rp, op = _res_orth(A, Wp, Zp, "s")
    print("dense %s n=%d fp32: mixed res %.3g orth %.3g | plain res %.3g orth %.3g (units of n eps)" % (
        kind, n, rm, om, rp, op))
    assert rm <= 1.0 and om <= 1.0
    assert om < op


def test_dense_index_range_and_host_buffers():
    import ctypes
    import paper_1304_1864_gb300 as m
    n = 200
    d, e = inputs.make("uniform_spectrum", n, seed=2)
    A = np.asfortranarray(_qtq(d, e, seed=3))
    W = np.zeros(21)
    Z = np.full((21, n + 5), np.nan)  # column-major n x 21 with ldz = n + 5
    mcount = ctypes.c_int(0)
    rc = m.mrrr_syev_d(n, A.ctypes.data_as(ctypes.c_void_p), n, m.MRRR_INDEX, ctypes.c_double(0),
                       ctypes.c_double(0), 90, 110, m.MRRR_MIXED, None, ctypes.byref(mcount),
                       W.ctypes.data_as(ctypes.c_void_p), Z.ctypes.data_as(ctypes.c_void_p), n + 5, None)
    assert rc == 0 and mcount.value == 21
    assert np.all(np.isnan(Z[:, n:]))
    hi, lo = oracle.eigvals(d, e, 90, 110)
    an = np.abs(A).sum(axis=0).max()
    assert np.max(np.abs(W - (hi + lo))) <= 2 * n * EPS["d"] * an
    Zc = Z[:, :n].T
    R = A @ Zc - Zc * W[None, :]
    assert np.linalg.norm(R, axis=0).max() <= n * EPS["d"] * an
