"""mrrr_eigvecs_noalloc_s: eigenvectors for given eigenvalues with no device
allocation.

This entry point is for callers that must not allocate device memory when
they call the solver: real-time or embedded hosts that reserve all their
memory at start-up, and libraries whose device memory belongs to another
framework's allocator.  Its scratch is one fixed device array inside
libmrrr.so.  The GPU test checks its eigenvectors against those of
mrrr_solve_s (the allocating entry point) on two calls in a row, with
different sizes, so that a call that depended on leftovers of the previous
one would fail.  The second call asks for an index range in the middle of
the spectrum, whose first and last eigenvalues take their gaps from the
eigenvalues just outside the range.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1304_1864_gb300 as m
from oracle import metrics
from paper_1304_1864_gb300 import inputs

from . import _acc


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_rejects_sizes_beyond_the_limit():
    # the size check comes before any CUDA call, so this runs without a GPU
    d = np.ones(4, np.float32)
    big = m.lib().mrrr_eigvecs_noalloc_s(1025, ctypes.c_void_p(d.ctypes.data), ctypes.c_void_p(d.ctypes.data), 1, 1,
                                         ctypes.c_void_p(d.ctypes.data), ctypes.c_void_p(d.ctypes.data), 1025, None)
    assert big == m.MRRR_ERR_ARG
    many = m.lib().mrrr_eigvecs_noalloc_s(4, ctypes.c_void_p(d.ctypes.data), ctypes.c_void_p(d.ctypes.data), 1, 1025,
                                          ctypes.c_void_p(d.ctypes.data), ctypes.c_void_p(d.ctypes.data), 4, None)
    assert many == m.MRRR_ERR_ARG


@pytest.mark.gpu
def test_noalloc_matches_solve_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    # the entry point needs eigenvalues separated by more than the mixed gaptol;
    # Clement (integer spectrum) and Hermite matrices have no clusters
    cases = [(inputs.clement(300), 1, 300),    # all eigenpairs of one matrix
             (inputs.hermite(700), 151, 350)]  # then a subset of a larger one
    for (d, e), il, iu in cases:
        n = d.size
        k = iu - il + 1
        dg = torch.tensor(d, dtype=torch.float32, device="cuda")
        eg = torch.tensor(e, dtype=torch.float32, device="cuda")
        # reference: the allocating solver on the same matrix and index range
        W, Z, st = m.solve(dg, eg, mode="mixed", range="index", il=il, iu=iu)
        assert st["status"] == 0 and st["nclusters"] == 0, "case needs well separated eigenvalues"
        Zn = torch.full((k, n), float("nan"), dtype=torch.float32, device="cuda")  # column-major n x k
        rc = m.mrrr_eigvecs_noalloc_s(n, _vp(dg), _vp(eg), il, k, _vp(W), _vp(Zn), n,
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0, m.strerror(rc)
        torch.cuda.synchronize()
        Zn = _acc.as_np(Zn.T)
        Wh = _acc.as_np(W).astype(np.float64)
        Zr = _acc.as_np(Z)
        d64, e64 = _acc.exact_input(d, e, "s")
        assert np.all(np.isfinite(Zn))
        # the same accuracy targets as every mixed-precision test
        _acc.check_res_orth(d64, e64, Wh, Zn, "s", "mixed")
        _acc.check_sign_convention(Zn, "s")
        # column by column against the allocating solver: both vectors lie within
        # ||r|| / gap of the true eigenvector (Gap Theorem), so their angle is at
        # most the sum of the two bounds
        r_n = metrics.residuals(d64, e64, Wh, Zn)[0]
        r_r = metrics.residuals(d64, e64, Wh, Zr)[0]
        hi, lo = oracle.eigvals(d64, e64)
        lam = hi + lo
        gaps = np.minimum(np.diff(lam, prepend=-np.inf), np.diff(lam, append=np.inf))[il - 1:iu]
        s = metrics.sin_angles(Zn.astype(np.float64), Zr.astype(np.float64))
        bound = (r_n + r_r) / gaps * 1.01 + 4 * 2.0 ** -24 * np.sqrt(n)
        assert np.all(s <= bound), "max excess %.3g" % np.max(s - bound)


@pytest.mark.gpu
def test_noalloc_rejects_host_pointers():
    d = np.linspace(-1, 1, 16).astype(np.float32)
    e = np.full(15, 0.3, np.float32)
    W = np.zeros(16, np.float32)
    Z = np.zeros((16, 16), np.float32)
    rc = m.lib().mrrr_eigvecs_noalloc_s(16, ctypes.c_void_p(d.ctypes.data), ctypes.c_void_p(e.ctypes.data), 1, 16,
                                        ctypes.c_void_p(W.ctypes.data), ctypes.c_void_p(Z.ctypes.data), 16, None)
    assert rc == m.MRRR_ERR_ARG
