"""Oracle for the symmetric tridiagonal eigenproblem -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The solver library neither imports nor
links anything here, and this package imports nothing from the solver.

The functions are thin ctypes wrappers over ``oracle.c`` (IEEE binary128):

* :func:`eigvals`  -- Sturm-sequence bisection on T (no LDL^T, no shifts).
* :func:`eigvecs`  -- inverse iteration + modified Gram-Schmidt.
* :func:`jacobi`   -- dense cyclic Jacobi (brute force for tiny inputs).
* :func:`residual_ortho` -- the accuracy measures R and O of Eq. (1.1).
* :mod:`oracle.metrics` -- the same measures for large n, with blocked
  double-double accumulation (numpy only).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        L.oracle_eigvals.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int]
        L.oracle_eigvals.restype = ctypes.c_int
        L.oracle_sturm_count.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_double]
        L.oracle_sturm_count.restype = ctypes.c_int
        L.oracle_eigvecs.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, dp, dp, dp, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_uint64]
        L.oracle_eigvecs.restype = ctypes.c_int
        L.oracle_jacobi.argtypes = [ctypes.c_int, dp, dp, dp, dp]
        L.oracle_jacobi.restype = ctypes.c_int
        L.oracle_residual_ortho.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, dp, dp, ctypes.c_int,
                                            dp, dp, dp, dp, ctypes.c_int]
        L.oracle_residual_ortho.restype = ctypes.c_int
        L.oracle_max_threads.argtypes = []
        L.oracle_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def max_threads() -> int:
    return lib().oracle_max_threads()


def eigvals(d, e, il=1, iu=None, nthreads=0):
    """Eigenvalues il..iu (1-based, inclusive) of T = tridiag(e, d, e).

    Returns ``(hi, lo)``: each eigenvalue is the unevaluated sum hi + lo of two
    doubles (the binary128 bisection midpoint)."""
    d = _f64(d)
    n = d.size
    e = _f64(e) if n > 1 else np.zeros(1)
    iu = n if iu is None else iu
    k = iu - il + 1
    hi = np.empty(max(k, 1))
    lo = np.empty(max(k, 1))
    rc = lib().oracle_eigvals(n, _p(d), _p(e), il, iu, _p(hi), _p(lo), nthreads)
    if rc != 0:
        raise ValueError("oracle_eigvals: bad arguments or non-finite input")
    return hi[:k], lo[:k]


def sturm_count(d, e, x_hi, x_lo=0.0) -> int:
    """Number of eigenvalues of T strictly below x = x_hi + x_lo."""
    d = _f64(d)
    e = _f64(e) if d.size > 1 else np.zeros(1)
    return lib().oracle_sturm_count(d.size, _p(d), _p(e), float(x_hi), float(x_lo))


def eigvecs(d, e, lam_hi, lam_lo=None, gs_window=1e-3, iters=3, seed=12345):
    """Unit eigenvectors (n x k, column-major in a Fortran-ordered array) for the
    eigenvalues lam_hi + lam_lo, by inverse iteration in binary128."""
    d = _f64(d)
    n = d.size
    e = _f64(e) if n > 1 else np.zeros(1)
    lam_hi = _f64(lam_hi)
    lam_lo = np.zeros_like(lam_hi) if lam_lo is None else _f64(lam_lo)
    k = lam_hi.size
    Z = np.zeros((n, max(k, 1)), dtype=np.float64, order="F")
    rc = lib().oracle_eigvecs(n, _p(d), _p(e), k, _p(lam_hi), _p(lam_lo), _p(Z), n,
                              float(gs_window), int(iters), int(seed))
    if rc != 0:
        raise ValueError("oracle_eigvecs: bad arguments")
    return Z[:, :k]


def jacobi(A):
    """Eigenvalues (hi, lo) and eigenvectors of a dense symmetric matrix by
    cyclic Jacobi in binary128 (brute force; meant for n <= 64)."""
    A = np.asfortranarray(np.asarray(A, dtype=np.float64))
    n = A.shape[0]
    hi = np.empty(n)
    lo = np.empty(n)
    V = np.zeros((n, n), dtype=np.float64, order="F")
    rc = lib().oracle_jacobi(n, _p(A), _p(hi), _p(lo), _p(V))
    if rc < 0:
        raise ValueError("oracle_jacobi: bad arguments")
    return hi, lo, V


def residual_ortho(d, e, W, Z, nthreads=0):
    """Eq. (1.1) in binary128: returns dict with per-column ``res`` (1-norm
    residual / ||T||_1), ``res2`` (2-norm residual), ``R`` = max res,
    ``O`` = max_{i!=j} |z_i^T z_j| and ``O_diag`` = max_j |z_j^T z_j - 1|."""
    d = _f64(d)
    n = d.size
    e = _f64(e) if n > 1 else np.zeros(1)
    W = _f64(W)
    Z = np.asfortranarray(np.asarray(Z, dtype=np.float64))
    k = W.size
    res = np.empty(max(k, 1))
    res2 = np.empty(max(k, 1))
    o = np.zeros(1)
    od = np.zeros(1)
    rc = lib().oracle_residual_ortho(n, _p(d), _p(e), k, _p(W), _p(Z), Z.shape[0] if k else n,
                                     _p(res), _p(res2), _p(o), _p(od), nthreads)
    if rc != 0:
        raise ValueError("oracle_residual_ortho: bad arguments")
    return {"res": res[:k], "res2": res2[:k], "R": float(res[:k].max()) if k else 0.0,
            "O": float(o[0]), "O_diag": float(od[0])}
