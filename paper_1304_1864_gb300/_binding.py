"""ctypes binding of the C ABI in include/mrrr.h (argument marshalling only).

Every step of the solve runs in the CUDA kernels of libmrrr.so; this module
only converts Python/torch/numpy arguments into pointers and sizes.  If the
library cannot be built or loaded, every call raises -- there is no CPU
fallback.
"""
import ctypes
import os

import numpy as np

from . import build as _build

MRRR_ALL, MRRR_INDEX, MRRR_VALUE = 0, 1, 2
MRRR_PLAIN, MRRR_MIXED = 0, 1
MRRR_OK, MRRR_ERR_ARG, MRRR_ERR_NONFINITE, MRRR_ERR_NOCONV = 0, -1, -2, -3
MRRR_ERR_NOMEM, MRRR_ERR_CUDA, MRRR_ERR_TIMEOUT, MRRR_ERR_NOREP = -4, -5, -6, -7
MRRR_ERR_CANCELLED = -8
MRRR_FLAG_NO_LOWPREC_BISECT, MRRR_FLAG_TIMING, MRRR_FLAG_STRICT_GROWTH, MRRR_FLAG_NO_TUNE = 1, 4, 8, 16
MRRR_FLAG_TEST_REJECT_CHILD, MRRR_FLAG_E_REP, MRRR_FLAG_RRR_TEST = 32, 64, 128
MRRR_FLAG_TEST_NO_REP = 256
NPHASES = 8
PHASES = ("prep", "root", "bisect", "classify", "shift", "refine", "rqi", "finish")


class MrrrStats(ctypes.Structure):
    _fields_ = [("nblocks", ctypes.c_int), ("d_max", ctypes.c_int), ("nclusters", ctypes.c_int),
                ("largest_cluster", ctypes.c_int), ("reps_failed", ctypes.c_int), ("rqi_iters", ctypes.c_int),
                ("fallbacks", ctypes.c_int), ("noconv", ctypes.c_int),
                ("qd_bisect", ctypes.c_longlong), ("qd_refine", ctypes.c_longlong), ("qd_rqi", ctypes.c_longlong),
                ("qd_shift", ctypes.c_longlong), ("qd_low", ctypes.c_longlong), ("verify_fail", ctypes.c_int),
                ("reps_relaxed", ctypes.c_int), ("rqi_warps_per_sm", ctypes.c_int),
                ("timed", ctypes.c_int), ("phase_launches", ctypes.c_int * NPHASES),
                ("phase_ms", ctypes.c_double * NPHASES), ("rqi_rows", ctypes.c_longlong),
                ("reps_backtracked", ctypes.c_int), ("reps_krr_relaxed", ctypes.c_int), ("krr_max", ctypes.c_double)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f not in ("phase_launches", "phase_ms")}
        d["phase_launches"] = dict(zip(PHASES, list(self.phase_launches)))
        d["phase_ms"] = dict(zip(PHASES, list(self.phase_ms)))
        return d


class MrrrParams(ctypes.Structure):
    _fields_ = [("gaptol", ctypes.c_double), ("xi", ctypes.c_double), ("krs", ctypes.c_double),
                ("max_depth", ctypes.c_int), ("max_rqi", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("flags", ctypes.c_int), ("stats", ctypes.POINTER(MrrrStats))]


MRRR_PENDING = 1


class MrrrServeConfig(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_int), ("max_batch", ctypes.c_int), ("hbm_budget", ctypes.c_longlong),
                ("alloc_failures", ctypes.c_int)]


class MrrrRequest(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("mode", ctypes.c_int), ("n", ctypes.c_int),
                ("d", ctypes.c_void_p), ("e", ctypes.c_void_p), ("il", ctypes.c_int), ("iu", ctypes.c_int),
                ("W", ctypes.c_void_p), ("Z", ctypes.c_void_p), ("ldz", ctypes.c_int),
                ("stream", ctypes.c_void_p)]


class MrrrServeInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("m", ctypes.c_int), ("batch", ctypes.c_int),
                ("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double)]


class MrrrServeStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_longlong), ("eigenpairs", ctypes.c_longlong), ("batches", ctypes.c_longlong),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("busy_s", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class MrrrError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__("%s: %s (status %d)" % (what or "mrrr", strerror(code), code))


_lib = None


def lib():
    """Load (building first if needed) libmrrr.so."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        for name, real in (("mrrr_solve_s", ctypes.c_float), ("mrrr_solve_d", ctypes.c_double)):
            f = getattr(L, name)
            f.argtypes = [ctypes.c_int, vp, vp, ctypes.c_int, real, real, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                          ctypes.POINTER(MrrrParams), ctypes.POINTER(ctypes.c_int), vp, vp, ctypes.c_int, vp]
            f.restype = ctypes.c_int
        for name in ("mrrr_solve_batch_s", "mrrr_solve_batch_d"):
            f = getattr(L, name)
            f.argtypes = [ctypes.c_int, vp, vp, vp, vp, vp, ctypes.c_int, ctypes.POINTER(MrrrParams), vp,
                          vp, vp, vp, vp, vp]
            f.restype = ctypes.c_int
        for name, real in (("mrrr_syev_s", ctypes.c_float), ("mrrr_syev_d", ctypes.c_double)):
            f = getattr(L, name)
            f.argtypes = [ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, real, real, ctypes.c_int, ctypes.c_int,
                          ctypes.c_int, ctypes.POINTER(MrrrParams), ctypes.POINTER(ctypes.c_int), vp, vp, ctypes.c_int,
                          vp]
            f.restype = ctypes.c_int
        for name in ("mrrr_partition_s", "mrrr_partition_d"):
            f = getattr(L, name)
            f.argtypes = [ctypes.c_int, vp, vp, ctypes.c_int, ctypes.POINTER(MrrrParams), ctypes.c_int, vp, vp, vp]
            f.restype = ctypes.c_int
        L.mrrr_eigvecs_noalloc_s.argtypes = [ctypes.c_int, vp, vp, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_int,
                                             vp]
        L.mrrr_eigvecs_noalloc_s.restype = ctypes.c_int
        L.mrrr_serve_open.argtypes = [ctypes.POINTER(MrrrServeConfig), ctypes.POINTER(ctypes.c_void_p)]
        L.mrrr_serve_submit.argtypes = [vp, ctypes.POINTER(MrrrRequest), ctypes.POINTER(ctypes.c_longlong)]
        L.mrrr_serve_poll.argtypes = [vp, ctypes.c_longlong, ctypes.c_int, ctypes.POINTER(MrrrServeInfo)]
        L.mrrr_serve_stats_get.argtypes = [vp, ctypes.POINTER(MrrrServeStats)]
        L.mrrr_serve_cancel.argtypes = [vp, ctypes.c_longlong]
        L.mrrr_serve_close.argtypes = [vp]
        for name in ("mrrr_serve_open", "mrrr_serve_submit", "mrrr_serve_poll", "mrrr_serve_stats_get",
                     "mrrr_serve_close"):
            getattr(L, name).restype = ctypes.c_int
        L.mrrr_probe_fp64_fma.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double), vp]
        L.mrrr_probe_fp64_fma.restype = ctypes.c_int
        L.mrrr_strerror.argtypes = [ctypes.c_int]
        L.mrrr_strerror.restype = ctypes.c_char_p
        L.mrrr_version.argtypes = []
        L.mrrr_version.restype = ctypes.c_char_p
        _lib = L
    return _lib


def strerror(code):
    try:
        return lib().mrrr_strerror(int(code)).decode()
    except Exception:  # library unavailable
        return "status %d" % code


# ------------------------------------------------------------------ C-ABI names

def mrrr_solve_s(n, d, e, rng, vl, vu, il, iu, mode, params, m_out, W, Z, ldz, stream):
    return lib().mrrr_solve_s(n, d, e, rng, vl, vu, il, iu, mode, params, m_out, W, Z, ldz, stream)


def mrrr_solve_d(n, d, e, rng, vl, vu, il, iu, mode, params, m_out, W, Z, ldz, stream):
    return lib().mrrr_solve_d(n, d, e, rng, vl, vu, il, iu, mode, params, m_out, W, Z, ldz, stream)


def mrrr_solve_batch_s(nb, n, d, e, il, iu, mode, params, m_out, W, Z, ldz, status, stream):
    return lib().mrrr_solve_batch_s(nb, n, d, e, il, iu, mode, params, m_out, W, Z, ldz, status, stream)


def mrrr_solve_batch_d(nb, n, d, e, il, iu, mode, params, m_out, W, Z, ldz, status, stream):
    return lib().mrrr_solve_batch_d(nb, n, d, e, il, iu, mode, params, m_out, W, Z, ldz, status, stream)


def mrrr_syev_s(n, A, lda, rng, vl, vu, il, iu, mode, params, m_out, W, Z, ldz, stream):
    return lib().mrrr_syev_s(n, A, lda, rng, vl, vu, il, iu, mode, params, m_out, W, Z, ldz, stream)


def mrrr_syev_d(n, A, lda, rng, vl, vu, il, iu, mode, params, m_out, W, Z, ldz, stream):
    return lib().mrrr_syev_d(n, A, lda, rng, vl, vu, il, iu, mode, params, m_out, W, Z, ldz, stream)


def mrrr_partition_s(n, d, e, mode, params, nparts, il, iu, stream):
    return lib().mrrr_partition_s(n, d, e, mode, params, nparts, il, iu, stream)


def mrrr_partition_d(n, d, e, mode, params, nparts, il, iu, stream):
    return lib().mrrr_partition_d(n, d, e, mode, params, nparts, il, iu, stream)


def mrrr_eigvecs_noalloc_s(n, d, e, il, k, W, Z, ldz, stream):
    return lib().mrrr_eigvecs_noalloc_s(n, d, e, il, k, W, Z, ldz, stream)


def mrrr_serve_open(cfg, out):
    return lib().mrrr_serve_open(cfg, out)


def mrrr_serve_submit(server, req, ticket):
    return lib().mrrr_serve_submit(server, req, ticket)


def mrrr_serve_poll(server, ticket, wait_ms, info):
    return lib().mrrr_serve_poll(server, ticket, wait_ms, info)


def mrrr_serve_cancel(server, ticket):
    return lib().mrrr_serve_cancel(server, ticket)


def mrrr_serve_stats_get(server, out):
    return lib().mrrr_serve_stats_get(server, out)


def mrrr_serve_close(server):
    return lib().mrrr_serve_close(server)


def mrrr_probe_fp64_fma(iters, gflops, ms, stream):
    return lib().mrrr_probe_fp64_fma(iters, gflops, ms, stream)


def probe_fp64(iters=0, stream=None):
    """Measured binary64 FMA throughput of the current device:
    (GFLOP/s, milliseconds of the timed launch)."""
    g = ctypes.c_double(0.0)
    t = ctypes.c_double(0.0)
    rc = mrrr_probe_fp64_fma(iters, ctypes.byref(g), ctypes.byref(t), _stream_handle(stream, True))
    if rc != MRRR_OK:
        raise MrrrError(rc, "mrrr_probe_fp64_fma")
    return g.value, t.value


def mrrr_strerror(code):
    return strerror(code)


def mrrr_version():
    return lib().mrrr_version().decode()


# ------------------------------------------------------------------ convenience

def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(x.ctypes.data)


def make_params(gaptol=0.0, xi=0.0, krs=0.0, max_depth=0, max_rqi=0, seed=0, flags=0, stats=None):
    p = MrrrParams()
    p.gaptol, p.xi, p.krs = gaptol, xi, krs
    p.max_depth, p.max_rqi, p.seed, p.flags = max_depth, max_rqi, seed, flags
    p.stats = ctypes.pointer(stats) if stats is not None else None
    return p


def _stream_handle(stream, device_side):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    if device_side:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


def solve(d, e, mode="mixed", range="all", vl=0.0, vu=0.0, il=1, iu=None, stream=None, timing=False,
          check=True, **param_kw):
    """Eigenpairs of the symmetric tridiagonal (d, e).

    d, e: torch tensors (CUDA or CPU) or numpy arrays, float32 (mrrr_solve_s) or
    float64 (mrrr_solve_d).  Returns (W, Z, stats) with Z of shape (n, m),
    column-major, on the same side as d.  mode: 'mixed' or 'plain';
    range: 'all', 'index' (il..iu, 1-based) or 'value' ((vl, vu])."""
    torch_in = _is_torch(d)
    n = int(d.shape[0])
    dt = d.dtype
    single = (str(dt).endswith("float32"))
    rng = {"all": MRRR_ALL, "index": MRRR_INDEX, "value": MRRR_VALUE}[range]
    iu = n if iu is None else iu
    k = (iu - il + 1) if rng == MRRR_INDEX else n
    kk = max(k, 1)
    if torch_in:
        import torch
        W = torch.empty(kk, dtype=d.dtype, device=d.device)
        Zt = torch.empty((kk, max(n, 1)), dtype=d.dtype, device=d.device)
        dev = d.is_cuda
    else:
        d = np.ascontiguousarray(d)
        e = np.ascontiguousarray(e) if e is not None else None
        W = np.empty(kk, dtype=d.dtype)
        Zt = np.empty((kk, max(n, 1)), dtype=d.dtype)
        dev = False
    stats = MrrrStats()
    prm = make_params(stats=stats, flags=(MRRR_FLAG_TIMING if timing else 0) | param_kw.pop("flags", 0), **param_kw)
    m = ctypes.c_int(0)
    fn = mrrr_solve_s if single else mrrr_solve_d
    real = ctypes.c_float if single else ctypes.c_double
    st = _stream_handle(stream, dev)
    rc = fn(n, _ptr(d), _ptr(e) if (e is not None and n > 1) else None, rng, real(vl), real(vu), il, iu,
            MRRR_MIXED if mode == "mixed" else MRRR_PLAIN, ctypes.byref(prm), ctypes.byref(m), _ptr(W), _ptr(Zt),
            max(n, 1), st)
    if check and rc not in (MRRR_OK, MRRR_ERR_NOCONV):
        raise MrrrError(rc, "mrrr_solve_" + ("s" if single else "d"))
    mm = m.value
    return W[:mm], Zt[:mm].T, stats.as_dict() | {"status": rc}


def solve_batch(mats, mode="mixed", ranges=None, stream=None, timing=False, check=True, **param_kw):
    """Solve independent tridiagonals in one batched call.  mats: list of
    (d, e) CUDA tensors, all float32 or all float64.  ranges: optional list
    of (il, iu).  Returns (list of (W, Z), stats, statuses)."""
    import torch
    nb = len(mats)
    single = mats[0][0].dtype == torch.float32
    ns = (ctypes.c_int * nb)(*[int(m[0].shape[0]) for m in mats])
    dp = (ctypes.c_void_p * nb)(*[m[0].data_ptr() for m in mats])
    ep = (ctypes.c_void_p * nb)(*[(m[1].data_ptr() if (m[1] is not None and m[1].numel() > 0) else 0) for m in mats])
    Ws, Zts = [], []
    for i, (dd, ee) in enumerate(mats):
        n = int(dd.shape[0])
        k = n if ranges is None else ranges[i][1] - ranges[i][0] + 1
        Ws.append(torch.empty(max(k, 1), dtype=dd.dtype, device=dd.device))
        Zts.append(torch.empty((max(k, 1), max(n, 1)), dtype=dd.dtype, device=dd.device))
    wp = (ctypes.c_void_p * nb)(*[w.data_ptr() for w in Ws])
    zp = (ctypes.c_void_p * nb)(*[z.data_ptr() for z in Zts])
    ld = (ctypes.c_int * nb)(*[max(int(m[0].shape[0]), 1) for m in mats])
    il = iu = None
    if ranges is not None:
        il = (ctypes.c_int * nb)(*[r[0] for r in ranges])
        iu = (ctypes.c_int * nb)(*[r[1] for r in ranges])
    mout = (ctypes.c_int * nb)()
    status = (ctypes.c_int * nb)()
    stats = MrrrStats()
    prm = make_params(stats=stats, flags=(MRRR_FLAG_TIMING if timing else 0) | param_kw.pop("flags", 0), **param_kw)
    fn = mrrr_solve_batch_s if single else mrrr_solve_batch_d
    st = _stream_handle(stream, True)
    rc = fn(nb, ctypes.cast(ns, ctypes.c_void_p), ctypes.cast(dp, ctypes.c_void_p), ctypes.cast(ep, ctypes.c_void_p),
            ctypes.cast(il, ctypes.c_void_p) if il is not None else None,
            ctypes.cast(iu, ctypes.c_void_p) if iu is not None else None,
            MRRR_MIXED if mode == "mixed" else MRRR_PLAIN, ctypes.byref(prm), ctypes.cast(mout, ctypes.c_void_p),
            ctypes.cast(wp, ctypes.c_void_p), ctypes.cast(zp, ctypes.c_void_p), ctypes.cast(ld, ctypes.c_void_p),
            ctypes.cast(status, ctypes.c_void_p), st)
    if check and rc not in (MRRR_OK, MRRR_ERR_NOCONV):
        raise MrrrError(rc, "mrrr_solve_batch")
    out = [(Ws[i][:mout[i]], Zts[i][:mout[i]].T) for i in range(nb)]
    return out, stats.as_dict() | {"status": rc}, list(status)


def solve_dense(A, mode="mixed", range="all", vl=0.0, vu=0.0, il=1, iu=None, stream=None, timing=False,
                check=True, **param_kw):
    """Eigenpairs of the dense symmetric matrix A (torch tensor or numpy
    array, float32 -> mrrr_syev_s, float64 -> mrrr_syev_d).  A is read in
    column-major order (for a symmetric matrix that is A itself).  Returns
    (W, Z, stats) with Z of shape (n, m) on the same side as A."""
    torch_in = _is_torch(A)
    n = int(A.shape[0])
    single = str(A.dtype).endswith("float32")
    rng = {"all": MRRR_ALL, "index": MRRR_INDEX, "value": MRRR_VALUE}[range]
    iu = n if iu is None else iu
    k = (iu - il + 1) if rng == MRRR_INDEX else n
    kk = max(k, 1)
    if torch_in:
        import torch
        A = A.contiguous()
        W = torch.empty(kk, dtype=A.dtype, device=A.device)
        Zt = torch.empty((kk, max(n, 1)), dtype=A.dtype, device=A.device)
        dev = A.is_cuda
    else:
        A = np.ascontiguousarray(A)
        W = np.empty(kk, dtype=A.dtype)
        Zt = np.empty((kk, max(n, 1)), dtype=A.dtype)
        dev = False
    stats = MrrrStats()
    prm = make_params(stats=stats, flags=(MRRR_FLAG_TIMING if timing else 0) | param_kw.pop("flags", 0), **param_kw)
    m = ctypes.c_int(0)
    fn = mrrr_syev_s if single else mrrr_syev_d
    real = ctypes.c_float if single else ctypes.c_double
    rc = fn(n, _ptr(A), max(n, 1), rng, real(vl), real(vu), il, iu, MRRR_MIXED if mode == "mixed" else MRRR_PLAIN,
            ctypes.byref(prm), ctypes.byref(m), _ptr(W), _ptr(Zt), max(n, 1), _stream_handle(stream, dev))
    if check and rc not in (MRRR_OK, MRRR_ERR_NOCONV):
        raise MrrrError(rc, "mrrr_syev_" + ("s" if single else "d"))
    mm = m.value
    return W[:mm], Zt[:mm].T, stats.as_dict() | {"status": rc}


def partition(d, e, nparts, mode="mixed", stream=None, **param_kw):
    """Index ranges (il, iu), 1-based inclusive, of nparts independent solves
    of the tridiagonal (d, e) (mrrr_partition_s / _d); an empty part has
    il = iu + 1."""
    n = int(d.shape[0])
    single = str(d.dtype).endswith("float32")
    dev = _is_torch(d) and d.is_cuda
    if not _is_torch(d):
        d = np.ascontiguousarray(d)
        e = np.ascontiguousarray(e) if e is not None else None
    il = (ctypes.c_int * nparts)()
    iu = (ctypes.c_int * nparts)()
    prm = make_params(**param_kw)
    fn = mrrr_partition_s if single else mrrr_partition_d
    rc = fn(n, _ptr(d), _ptr(e) if (e is not None and n > 1) else None, MRRR_MIXED if mode == "mixed" else MRRR_PLAIN,
            ctypes.byref(prm), nparts, ctypes.cast(il, ctypes.c_void_p), ctypes.cast(iu, ctypes.c_void_p),
            _stream_handle(stream, dev))
    if rc != MRRR_OK:
        raise MrrrError(rc, "mrrr_partition")
    return list(zip(list(il), list(iu)))


class Server:
    """The serving loop (mrrr_serve_*).  submit() takes numpy or torch arrays
    for d and e and the output arrays W (>= k values) and Z (k x n, i.e. the
    column-major n x k result, row-major in Python); the arrays are kept
    referenced until the ticket is polled.  poll() returns (status, info dict)
    or None while the request is pending."""

    def __init__(self, workers=0, max_batch=0, hbm_budget=0, alloc_failures=0):
        self._h = ctypes.c_void_p()
        cfg = MrrrServeConfig(workers, max_batch, hbm_budget, alloc_failures)
        rc = lib().mrrr_serve_open(ctypes.byref(cfg), ctypes.byref(self._h))
        if rc != MRRR_OK:
            raise MrrrError(rc, "mrrr_serve_open")
        self._keep = {}

    def submit(self, d, e, W, Z, mode="mixed", il=0, iu=0, stream=None):
        n = int(d.shape[0])
        prec = 0 if str(d.dtype).endswith("float32") else 1
        on_dev = any(_is_torch(x) and x.is_cuda for x in (d, W))
        req = MrrrRequest(prec, MRRR_MIXED if mode == "mixed" else MRRR_PLAIN, n, _ptr(d),
                          _ptr(e) if n > 1 else None, il, iu, _ptr(W), _ptr(Z), n,
                          _stream_handle(stream, on_dev) if on_dev else None)
        t = ctypes.c_longlong(0)
        rc = lib().mrrr_serve_submit(self._h, ctypes.byref(req), ctypes.byref(t))
        if rc != MRRR_OK:
            raise MrrrError(rc, "mrrr_serve_submit")
        self._keep[t.value] = (d, e, W, Z)
        return t.value

    def poll(self, ticket, wait_ms=-1):
        info = MrrrServeInfo()
        rc = lib().mrrr_serve_poll(self._h, ticket, wait_ms, ctypes.byref(info))
        if rc == MRRR_PENDING:
            return None
        if rc == MRRR_ERR_ARG and ticket not in self._keep:
            raise MrrrError(rc, "mrrr_serve_poll")
        self._keep.pop(ticket, None)
        return rc, {f: getattr(info, f) for f, _ in info._fields_}

    def cancel(self, ticket):
        """MRRR_OK if the request was withdrawn before it ran, MRRR_PENDING if
        it was already admitted (poll it)."""
        rc = lib().mrrr_serve_cancel(self._h, ticket)
        if rc == MRRR_ERR_ARG:
            raise MrrrError(rc, "mrrr_serve_cancel")
        return rc

    def stats(self):
        st = MrrrServeStats()
        rc = lib().mrrr_serve_stats_get(self._h, ctypes.byref(st))
        if rc != MRRR_OK:
            raise MrrrError(rc, "mrrr_serve_stats_get")
        return st.as_dict()

    def close(self):
        if self._h:
            lib().mrrr_serve_close(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
