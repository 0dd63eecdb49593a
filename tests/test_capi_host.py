"""Host-side checks of the C ABI (no GPU needed): the library builds and
exports every entry point declared in include/*.h, the statistics struct
of the binding matches the header, and invalid arguments are rejected before
any device work."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1304_1864_gb300 as m

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mrrr.h")


def _declared_functions():
    names = set()
    inc = os.path.dirname(HEADER)
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            src = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, f)).read(), flags=re.S)
            names |= set(re.findall(r"\b(mrrr_\w+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = m.lib()
    names = _declared_functions()
    assert {"mrrr_solve_s", "mrrr_solve_d", "mrrr_solve_batch_s", "mrrr_solve_batch_d", "mrrr_strerror",
            "mrrr_probe_fp64_fma"} <= set(names)
    for name in names:
        assert hasattr(L, name), "libmrrr.so does not export " + name


def test_stats_struct_matches_header():
    src = open(HEADER).read()
    body = src.split("} mrrr_stats;")[0].rsplit("typedef struct {", 1)[1]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"(int|long long|double)\s+(\w+)(\[\w+\])?;", body)
    names = [f[1] for f in fields]
    assert names == [f for f, _ in m.MrrrStats._fields_]
    sizes = {"int": 4, "long long": 8, "double": 8}
    for (ctype, name, arr), (fname, ftype) in zip(fields, m.MrrrStats._fields_):
        n = 8 if arr else 1
        assert ctypes.sizeof(ftype) == sizes[ctype] * n, name


def test_params_struct_matches_header():
    src = open(HEADER).read()
    body = src.split("} mrrr_params;")[0].rsplit("typedef struct {", 1)[1]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"(?:double|int|uint64_t|mrrr_stats\*)\s+(\w+);", body)
    assert names == [f for f, _ in m.MrrrParams._fields_]


def _call_s(n, d, e, rng=0, vl=0.0, vu=0.0, il=1, iu=1, mode=1, W=True, Z=True, ldz=None):
    dp = ctypes.c_void_p(d.ctypes.data) if d is not None else None
    ep = ctypes.c_void_p(e.ctypes.data) if e is not None else None
    Wb = np.zeros(max(n, 1), np.float32)
    Zb = np.zeros((max(n, 1), max(n, 1)), np.float32)
    mc = ctypes.c_int(-7)
    rc = m.mrrr_solve_s(n, dp, ep, rng, ctypes.c_float(vl), ctypes.c_float(vu), il, iu, mode, None,
                        ctypes.byref(mc), ctypes.c_void_p(Wb.ctypes.data) if W else None,
                        ctypes.c_void_p(Zb.ctypes.data) if Z else None, n if ldz is None else ldz, None)
    return rc, mc.value


def test_invalid_arguments_rejected_without_device_work():
    d = np.ones(5, np.float32)
    e = np.ones(4, np.float32)
    assert _call_s(-1, d, e)[0] == m.MRRR_ERR_ARG
    assert _call_s(5, None, e)[0] == m.MRRR_ERR_ARG
    assert _call_s(5, d, None)[0] == m.MRRR_ERR_ARG
    assert _call_s(5, d, e, W=False)[0] == m.MRRR_ERR_ARG
    assert _call_s(5, d, e, ldz=4)[0] == m.MRRR_ERR_ARG
    assert _call_s(5, d, e, rng=1, il=0, iu=3)[0] == m.MRRR_ERR_ARG
    assert _call_s(5, d, e, rng=1, il=4, iu=3)[0] == m.MRRR_ERR_ARG
    assert _call_s(5, d, e, rng=1, il=1, iu=6)[0] == m.MRRR_ERR_ARG
    assert _call_s(5, d, e, rng=2, vl=1.0, vu=1.0)[0] == m.MRRR_ERR_ARG
    assert _call_s(5, d, e, rng=7)[0] == m.MRRR_ERR_ARG
    assert _call_s(5, d, e, mode=3)[0] == m.MRRR_ERR_ARG
    # n = 0 is a valid empty problem
    assert _call_s(0, d, e) == (0, 0)


def test_batch_invalid_arguments():
    rc = m.mrrr_solve_batch_s(-1, None, None, None, None, None, 1, None, None, None, None, None, None, None)
    assert rc == m.MRRR_ERR_ARG
    rc = m.mrrr_solve_batch_s(2, None, None, None, None, None, 1, None, None, None, None, None, None, None)
    assert rc == m.MRRR_ERR_ARG


def test_no_cpu_fallback():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present; the device path is covered by the gpu tests")
    d = np.linspace(-1, 1, 8).astype(np.float32)
    e = np.full(7, 0.5, np.float32)
    rc, _ = _call_s(8, d, e)
    assert rc == m.MRRR_ERR_CUDA
    with pytest.raises(m.MrrrError):
        m.solve(d, e)


def test_strerror_and_version():
    assert m.strerror(0) == "success"
    assert "argument" in m.strerror(m.MRRR_ERR_ARG)
    assert m.strerror(12345) == "unknown status"
    assert "sm_103a" in m.mrrr_version()


def _struct_fields(name):
    src = open(HEADER).read()
    body = src.split("} %s;" % name)[0].rsplit("typedef struct {", 1)[1]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        ctype, names = re.match(r"((?:const\s+)?(?:long long|int|double|void\*|mrrr_mode))\s+(.*)", decl).groups()
        for nm in names.split(","):
            out.append((ctype, nm.strip()))
    return out


@pytest.mark.parametrize("cname,pyname", [("mrrr_serve_config", "MrrrServeConfig"), ("mrrr_request", "MrrrRequest"),
                                          ("mrrr_serve_info", "MrrrServeInfo"), ("mrrr_serve_stats", "MrrrServeStats")])
def test_serve_structs_match_header(cname, pyname):
    fields = _struct_fields(cname)
    py = getattr(m, pyname)
    assert [n for _, n in fields] == [f for f, _ in py._fields_]
    sizes = {"int": 4, "mrrr_mode": 4, "long long": 8, "double": 8, "void*": 8, "const void*": 8}
    for (ctype, nm), (fname, ftype) in zip(fields, py._fields_):
        assert ctypes.sizeof(ftype) == sizes[ctype], nm


def test_serve_arguments_rejected_without_device_work():
    L = m.lib()
    t = ctypes.c_longlong(0)
    req = m.MrrrRequest()
    assert L.mrrr_serve_submit(None, ctypes.byref(req), ctypes.byref(t)) == m.MRRR_ERR_ARG
    assert L.mrrr_serve_poll(None, 1, 0, None) == m.MRRR_ERR_ARG
    assert L.mrrr_serve_stats_get(None, None) == m.MRRR_ERR_ARG
    assert L.mrrr_serve_cancel(None, 1) == m.MRRR_ERR_ARG
    assert L.mrrr_serve_close(None) == m.MRRR_ERR_ARG
    assert L.mrrr_serve_open(None, None) == m.MRRR_ERR_ARG
    bad = m.MrrrServeConfig(-1, 0, 0, 0)
    h = ctypes.c_void_p()
    assert L.mrrr_serve_open(ctypes.byref(bad), ctypes.byref(h)) == m.MRRR_ERR_ARG


def test_serve_open_without_device_fails_loudly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    h = ctypes.c_void_p()
    assert m.lib().mrrr_serve_open(None, ctypes.byref(h)) == m.MRRR_ERR_CUDA
