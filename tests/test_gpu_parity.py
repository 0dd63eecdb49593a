"""GPU parity: the CUDA solver through the C ABI against the binary128 oracle."""
import numpy as np
import pytest

from paper_1304_1864_gb300 import inputs

from . import _acc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MODES = [("s", "mixed"), ("d", "mixed"), ("s", "plain"), ("d", "plain")]


def _solve(d, e, prec, mode, **kw):
    import paper_1304_1864_gb300 as m
    dt = torch.float32 if prec == "s" else torch.float64
    dg = torch.tensor(np.asarray(d), dtype=dt, device="cuda")
    eg = torch.tensor(np.asarray(e), dtype=dt, device="cuda")
    W, Z, st = m.solve(dg, eg, mode=mode, **kw)
    torch.cuda.synchronize()
    return _acc.as_np(W), _acc.as_np(Z), st


def _full_check(d, e, prec, mode, vectors=True, **kw):
    d64, e64 = _acc.exact_input(d, e, prec)
    W, Z, st = _solve(d, e, prec, mode, **kw)
    assert st["status"] == 0, st
    assert W.size == d64.size
    assert np.all(np.diff(W) >= 0), "W not ascending"
    _acc.check_eigvals(d64, e64, W, prec, mode)
    res, orth = _acc.check_res_orth(d64, e64, W, Z, prec, mode)
    _acc.check_sign_convention(Z, prec)
    if vectors and d64.size <= 400:
        _acc.check_vectors_gap_theorem(d64, e64, W, Z, prec)
    return W, Z, st


@pytest.mark.parametrize("prec,mode", MODES)
@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 129, 300])
@pytest.mark.parametrize("kind", ["uniform", "121", "wilkinson", "clement", "glued"])
def test_small_sizes(kind, n, prec, mode):
    # sizes across one and several warps of eigenpairs, with ragged tails
    if kind == "glued" and n < 21:
        pytest.skip("glued needs n >= 21")
    d, e = inputs.make(kind, n, seed=n)
    _full_check(d, e, prec, mode)


@pytest.mark.parametrize("mode", ["plain", "mixed"])
def test_config_n500_uniform_fp64(mode):
    # one tridiagonal, n = 500, d, e ~ U(-1, 1) from seed 0, binary64 in/out
    d, e = inputs.workload_c1()[0]
    W, Z, st = _full_check(d, e, "d", mode, vectors=False)
    # every vector against the oracle through the Gap Theorem
    assert _acc.check_vectors_gap_theorem(d, e, W, Z, "d", idx=np.arange(0, 500, 7)) > 40


C2_NAMES = ("121", "wilkinson", "clement")


def _c2_oracle(i, d64, e64):
    return _acc.oracle_all("c2-" + C2_NAMES[i], d64, e64)


def test_config_n4001_mixed_single_double():
    # three matrices at n = 4001, each solved on its own, float32 in/out; every
    # eigenvalue against the oracle
    for i, (d, e) in enumerate(inputs.workload_c2()):
        d64, e64 = _acc.exact_input(d, e, "s")
        n = d64.size
        W, Z, st = _solve(d, e, "s", "mixed")
        assert st["status"] == 0 and W.size == n
        assert np.all(np.diff(W) >= 0)
        _acc.check_eigvals_all(d64, e64, W, "s", "mixed", _c2_oracle(i, d64, e64))
        _acc.check_res_orth(d64, e64, W, Z, "s", "mixed")
        _acc.check_sign_convention(Z, "s")


def test_config_n4001_batched_call():
    # the benchmark's launch configuration: the three n = 4001 matrices in one
    # mrrr_solve_batch_s call.  Each matrix's eigenpairs are bit-identical to
    # its own solve, and all 3 x 4001 eigenvalues are checked against the
    # oracle element by element.
    import paper_1304_1864_gb300 as m
    mats_h = inputs.workload_c2()
    mats = [(torch.tensor(d, dtype=torch.float32, device="cuda"), torch.tensor(e, dtype=torch.float32, device="cuda"))
            for d, e in mats_h]
    out, st, status = m.solve_batch(mats, mode="mixed")
    torch.cuda.synchronize()
    assert all(s == 0 for s in status), status
    for i, ((d, e), (dg, eg), (Wb, Zb)) in enumerate(zip(mats_h, mats, out)):
        W1, Z1, _ = m.solve(dg, eg, mode="mixed")
        assert torch.equal(W1, Wb) and torch.equal(Z1, Zb)
        d64, e64 = _acc.exact_input(d, e, "s")
        _acc.check_eigvals_all(d64, e64, _acc.as_np(Wb), "s", "mixed", _c2_oracle(i, d64, e64))


def test_config_n4001_batched_call_host_buffers():
    # the same call with every buffer in host memory (the end-to-end path):
    # the library stages inputs and outputs, results bit-identical to the
    # device-buffer call
    import ctypes
    import paper_1304_1864_gb300 as m
    mats_h = [(np.asarray(d, np.float32), np.asarray(e, np.float32)) for d, e in inputs.workload_c2()]
    mats = [(torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda()) for d, e in mats_h]
    out, st, status = m.solve_batch(mats, mode="mixed")
    nb = len(mats_h)
    n = [d.size for d, _ in mats_h]
    Wh = [np.full(k, np.nan, np.float32) for k in n]
    Zh = [np.full((k, k + 3), np.nan, np.float32) for k in n]  # leading dimension n + 3
    vp = ctypes.c_void_p

    def arr(t, xs):
        return ctypes.cast((t * nb)(*xs), vp)

    status_h = (ctypes.c_int * nb)()
    mout = (ctypes.c_int * nb)()
    rc = m.mrrr_solve_batch_s(nb, arr(ctypes.c_int, n), arr(vp, [d.ctypes.data for d, _ in mats_h]),
                              arr(vp, [e.ctypes.data for _, e in mats_h]), None, None, m.MRRR_MIXED, None,
                              ctypes.cast(mout, vp), arr(vp, [w.ctypes.data for w in Wh]),
                              arr(vp, [z.ctypes.data for z in Zh]), arr(ctypes.c_int, [k + 3 for k in n]),
                              ctypes.cast(status_h, vp), None)
    assert rc == 0 and list(status_h) == [0] * nb and list(mout) == n
    for (W, Z), w, z, k in zip(out, Wh, Zh, n):
        assert np.array_equal(_acc.as_np(W), w)
        assert np.array_equal(_acc.as_np(Z), z[:, :k].T)
        assert np.all(np.isnan(z[:, k:])), "padding rows beyond n were written"


def test_121_closed_form_full_size():
    # 1-2-1 at n = 4001: lambda_k = 2 - 2 cos(k pi/(n+1)), sine eigenvectors
    n = 4001
    d, e = inputs.one_two_one(n)
    W, Z, st = _solve(d, e, "s", "mixed")
    k = np.arange(1, n + 1)
    lam = 2 - 2 * np.cos(k * np.pi / (n + 1))
    assert np.max(np.abs(W - lam)) <= 2 * n * 2.0 ** -24 * 4
    cols = np.arange(0, n, 97)
    i = np.arange(1, n + 1)[:, None]
    zx = np.sqrt(2.0 / (n + 1)) * np.sin(i * (cols[None, :] + 1) * np.pi / (n + 1))
    gaps = np.minimum(np.diff(lam, prepend=-np.inf), np.diff(lam, append=np.inf))[cols]
    from oracle import metrics
    s = metrics.sin_angles(Z[:, cols].astype(np.float64), zx)
    # Gap theorem: sin <= ||r|| / gap, ||r|| <= n eps ||T|| (mixed target)
    assert np.all(s <= n * 2.0 ** -24 * 4 / gaps + 1e-6)


def test_clement_integer_spectrum_full_size():
    n = 4001
    d, e = inputs.clement(n)
    W, Z, st = _solve(d, e, "s", "mixed")
    exact = np.arange(-(n - 1), n, 2, dtype=np.float64)
    d64, e64 = _acc.exact_input(d, e, "s")
    from oracle import metrics
    # input rounding to float32 moves eigenvalues by <= 2 max|de| <= 2 eps_s max e
    bound = 2 * n * 2.0 ** -24 * metrics.tnorm1(d64, e64) + 2 * 2.0 ** -24 * e.max()
    assert np.max(np.abs(W - exact)) <= bound


def test_config_glued_wilkinson_mixed_double():
    # 40 copies of W_201 glued by 1e-8 (n = 8040), binary64 in/out,
    # double-double inside; all 8040 eigenvalues against the oracle
    d, e = inputs.workload_c3()[0]
    n = d.size
    W, Z, st = _solve(d, e, "d", "mixed")
    assert st["status"] == 0 and W.size == n
    assert np.all(np.diff(W) >= 0)
    _acc.check_eigvals_all(d, e, W, "d", "mixed", _acc.oracle_all("c3", d, e))
    _acc.check_res_orth(d, e, W, Z, "d", "mixed")


@pytest.mark.parametrize("prec", ["s", "d"])
def test_index_and_value_ranges(prec):
    n = 300
    d, e = inputs.uniform_random(n, 5)
    d64, e64 = _acc.exact_input(d, e, prec)
    for il, iu in [(1, 1), (1, 10), (150, 160), (291, 300), (1, 300), (37, 37)]:
        W, Z, st = _solve(d, e, prec, "mixed", range="index", il=il, iu=iu)
        assert W.size == iu - il + 1
        _acc.check_eigvals(d64, e64, W, prec, "mixed", il=il)
        _acc.check_res_orth(d64, e64, W, Z, prec, "mixed")
    import oracle
    hi, lo = oracle.eigvals(d64, e64)
    lam = hi + lo
    for vl, vu in [(-0.5, 0.25), (lam[10] - 1e-3, lam[20] + 1e-3), (-10.0, 10.0), (5.0, 6.0)]:
        W, Z, st = _solve(d, e, prec, "mixed", range="value", vl=vl, vu=vu)
        sel = np.nonzero((lam > vl) & (lam <= vu))[0]
        assert W.size == sel.size
        if sel.size:
            _acc.check_eigvals(d64, e64, W, prec, "mixed", il=int(sel[0]) + 1)
            _acc.check_res_orth(d64, e64, W, Z, prec, "mixed")


@pytest.mark.parametrize("prec", ["s", "d"])
def test_split_matrix_with_tied_blocks(prec):
    # glued W_21 copies with coupling 1e-20 split into identical blocks (exact
    # ties across blocks); W must still be ascending and Z orthonormal
    d, e = inputs.glued_wilkinson(6, 21, 1e-20)
    W, Z, st = _full_check(d, e, prec, "mixed", vectors=False)
    assert st["nblocks"] == 6


def test_split_many_identical_blocks_fp32():
    # 120 glued W_21 copies with coupling 1e-8: below the fp32 split threshold
    # (eps_x ||T||), so the matrix splits into 120 identical blocks whose
    # eigenvalues tie 120-fold; the final values come out in a rounding-
    # dependent order and are put in ascending order with their columns
    d, e = inputs.glued_wilkinson(120, 21, 1e-8)
    W, Z, st = _full_check(d, e, "s", "mixed", vectors=False)
    assert st["nblocks"] == 120
    assert np.all(np.diff(W) >= 0)


@pytest.mark.parametrize("prec", ["s", "d"])
def test_degenerate_inputs(prec):
    # diagonal matrix (every block of size 1), zero matrix, n = 1
    d = np.array([3.0, -1.0, 2.0, 2.0, 0.5])
    e = np.zeros(4)
    W, Z, st = _solve(d, e, prec, "mixed")
    assert np.allclose(W, np.sort(d))
    # each column is a signed unit coordinate vector
    assert np.all(np.abs(Z).max(axis=0) == 1.0) and np.all(np.abs(Z).sum(axis=0) == 1.0)
    assert np.all(Z.max(axis=0) == 1.0)
    W, Z, st = _solve(np.zeros(7), np.zeros(6), prec, "mixed")
    assert np.all(W == 0)
    _acc.check_res_orth(np.zeros(7), np.zeros(6), W, Z, prec, "mixed")
    W, Z, st = _solve(np.array([-4.5]), np.zeros(0), prec, "mixed")
    assert W[0] == -4.5 and Z[0, 0] == 1.0


def test_nonfinite_input_is_an_error():
    import paper_1304_1864_gb300 as m
    d = torch.tensor([1.0, float("nan"), 2.0], dtype=torch.float64, device="cuda")
    e = torch.tensor([1.0, 1.0], dtype=torch.float64, device="cuda")
    with pytest.raises(m.MrrrError) as ex:
        m.solve(d, e)
    assert ex.value.code == m.MRRR_ERR_NONFINITE


@pytest.mark.parametrize("prec", ["s", "d"])
def test_host_buffers_and_leading_dimension(prec):
    import ctypes
    import paper_1304_1864_gb300 as m
    n, ldz = 50, 64
    d, e = inputs.uniform_random(n, 2)
    dt = np.float32 if prec == "s" else np.float64
    d = d.astype(dt)
    e = e.astype(dt)
    W = np.zeros(n, dtype=dt)
    Z = np.full((n, ldz), 7.0, dtype=dt)  # row p = column p of a column-major n x ldz... layout
    mcount = ctypes.c_int(0)
    fn = m.mrrr_solve_s if prec == "s" else m.mrrr_solve_d
    real = ctypes.c_float if prec == "s" else ctypes.c_double
    rc = fn(n, d.ctypes.data_as(ctypes.c_void_p), e.ctypes.data_as(ctypes.c_void_p), 0, real(0), real(0), 1, n,
            1, None, ctypes.byref(mcount), W.ctypes.data_as(ctypes.c_void_p), Z.ctypes.data_as(ctypes.c_void_p),
            ldz, None)
    assert rc == 0 and mcount.value == n
    Zc = Z[:, :n].T  # column j of the column-major result is row j of Z
    assert np.all(Z[:, n:] == 7.0), "padding rows beyond n were written"
    d64, e64 = _acc.exact_input(d, e, prec)
    _acc.check_eigvals(d64, e64, W, prec, "mixed")
    _acc.check_res_orth(d64, e64, W, Zc, prec, "mixed")


@pytest.mark.parametrize("prec", ["s", "d"])
def test_batch_equals_individual(prec):
    import paper_1304_1864_gb300 as m
    dt = torch.float32 if prec == "s" else torch.float64
    mats = []
    for kind, n in [("uniform", 40), ("121", 77), ("wilkinson", 31), ("glued", 63), ("uniform", 1), ("clement", 90)]:
        d, e = inputs.make(kind, n, seed=n)
        mats.append((torch.tensor(d, dtype=dt, device="cuda"), torch.tensor(e, dtype=dt, device="cuda")))
    out, st, status = m.solve_batch(mats, mode="mixed")
    assert all(s == 0 for s in status)
    for (dd, ee), (Wb, Zb) in zip(mats, out):
        W1, Z1, _ = m.solve(dd, ee, mode="mixed")
        assert torch.equal(W1, Wb) and torch.equal(Z1, Zb)


def test_batched_workload_subsample():
    # independent tridiagonals of uneven size and type in one batched call:
    # n log-uniform in [32, 2048], types {U(-1,1), 1-2-1, Wilkinson, glued W_21}
    import paper_1304_1864_gb300 as m
    batch = inputs.workload_c4(count=48, seed=4)
    mats = [(torch.tensor(d, dtype=torch.float32, device="cuda"), torch.tensor(e, dtype=torch.float32, device="cuda"))
            for _, d, e in batch]
    out, st, status = m.solve_batch(mats, mode="mixed")
    assert all(s == 0 for s in status), status
    rng = np.random.default_rng(7)
    for (kind, d, e), (W, Z) in zip(batch, out):
        d64, e64 = _acc.exact_input(d, e, "s")
        W = _acc.as_np(W)
        Z = _acc.as_np(Z)
        n = d64.size
        assert W.size == n and np.all(np.diff(W) >= 0)
        idx = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 6)]))
        _acc.check_eigvals(d64, e64, W, "s", "mixed", idx=idx)
        _acc.check_res_orth(d64, e64, W, Z, "s", "mixed")


def test_rqi_grid_autotuner_does_not_change_results():
    # a batch large enough for the RQI grid to be tuned (more root singletons
    # than 152 SMs x 4 warps x 32 lanes): the first solves of a workload class
    # try each candidate grid, and every solve must return the same bits
    import paper_1304_1864_gb300 as m
    mats = []
    for j in range(64):
        d, e = inputs.make(("uniform", "121", "clement")[j % 3], 561, seed=900 + j)
        mats.append((torch.tensor(d, dtype=torch.float32, device="cuda"), torch.tensor(e, dtype=torch.float32,
                                                                                       device="cuda")))
    ref, st0, status = m.solve_batch(mats, mode="mixed", flags=m.MRRR_FLAG_NO_TUNE)
    assert all(s == 0 for s in status)
    assert st0["rqi_warps_per_sm"] == 16
    seen = set()
    for _ in range(5):
        out, st, status = m.solve_batch(mats, mode="mixed")
        assert all(s == 0 for s in status)
        seen.add(st["rqi_warps_per_sm"])
        for (W0, Z0), (W1, Z1) in zip(ref, out):
            assert torch.equal(W0, W1) and torch.equal(Z0, Z1)
    assert seen <= {16, 8, 4} and len(seen) >= 2
