"""The serving loop (mrrr_serve_*): requests of both precisions and modes, all
pairs or an index range, host or device buffers, submitted together so that
they are batched; every result must be the same as the same request solved
alone (mrrr_solve_s / mrrr_solve_d), and meet the accuracy targets.  Also:
admission under a tiny device budget (every request runs alone), continuous
batching while requests keep arriving, and the latency counters."""
import numpy as np
import pytest

from paper_1304_1864_gb300 import inputs

from . import _acc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (kind, n, precision, mode, il, iu, buffers on the device)
REQUESTS = [
    ("uniform", 300, "s", "mixed", 0, 0, True),
    ("121", 257, "s", "mixed", 0, 0, False),
    ("wilkinson", 201, "s", "mixed", 0, 0, True),
    ("uniform", 500, "s", "mixed", 51, 100, False),
    ("glued", 126, "s", "mixed", 0, 0, True),
    ("uniform", 200, "s", "plain", 0, 0, False),
    ("uniform", 120, "d", "mixed", 0, 0, True),
    ("clement", 97, "d", "mixed", 10, 30, False),
    ("uniform", 150, "d", "plain", 0, 0, True),
    ("uniform", 1, "s", "mixed", 0, 0, False),
]


def _make(kind, n, prec, mode, il, iu, on_dev, seed):
    import paper_1304_1864_gb300 as m
    d, e = inputs.make(kind, n, seed=seed)
    n = d.size
    npdt = np.float32 if prec == "s" else np.float64
    k = (iu - il + 1) if il else n
    if on_dev:
        tdt = torch.float32 if prec == "s" else torch.float64
        dd = torch.tensor(d, dtype=tdt, device="cuda")
        ee = torch.tensor(e if n > 1 else np.zeros(1), dtype=tdt, device="cuda")
        W = torch.full((k,), float("nan"), dtype=tdt, device="cuda")
        Z = torch.full((k, n), float("nan"), dtype=tdt, device="cuda")
    else:
        dd = d.astype(npdt)
        ee = (e if n > 1 else np.zeros(1)).astype(npdt)
        W = np.full(k, np.nan, npdt)
        Z = np.full((k, n), np.nan, npdt)
    # the same request solved alone
    kw = dict(range="index", il=il, iu=iu) if il else {}
    dref = torch.tensor(d, dtype=torch.float32 if prec == "s" else torch.float64, device="cuda")
    eref = torch.tensor(e if n > 1 else np.zeros(1), dtype=dref.dtype, device="cuda")
    W1, Z1, st = m.solve(dref, eref, mode=mode, **kw)
    assert st["status"] == 0
    return (d, e, dd, ee, W, Z), (_acc.as_np(W1), _acc.as_np(Z1))


def test_served_results_equal_alone():
    import paper_1304_1864_gb300 as m
    cases = [_make(*r, seed=11 + i) for i, r in enumerate(REQUESTS)]
    with m.Server(workers=2) as srv:
        tickets = []
        for (kind, n, prec, mode, il, iu, on_dev), ((d, e, dd, ee, W, Z), _) in zip(REQUESTS, cases):
            tickets.append(srv.submit(dd, ee, W, Z, mode=mode, il=il, iu=iu))
        infos = [srv.poll(t, wait_ms=-1) for t in tickets]
        stats = srv.stats()
    assert all(rc == 0 for rc, _ in infos), infos
    batched = max(info["batch"] for _, info in infos)
    assert batched > 1, "requests submitted together were never batched"
    for (kind, n, prec, mode, il, iu, on_dev), ((d, e, dd, ee, W, Z), (W1, Z1)), (_, info) in zip(REQUESTS, cases,
                                                                                                  infos):
        Wn, Zn = _acc.as_np(W), _acc.as_np(Z).T  # Z was k x n row-major = n x k column-major
        assert info["m"] == W1.size
        # the same computation in the mix as alone: identical bits
        assert np.array_equal(Wn, W1) and np.array_equal(Zn, Z1), (kind, n, prec, mode)
        d64, e64 = _acc.exact_input(d, e, prec)
        _acc.check_res_orth(d64, e64, Wn.astype(np.float64), Zn, prec, mode)
    assert stats["completed"] == len(REQUESTS)
    assert stats["p50_ms"] <= stats["p99_ms"] <= stats["max_ms"]
    assert stats["eigenpairs"] == sum(W1.size for _, (W1, _) in cases)


def test_tiny_budget_runs_each_request_alone():
    import paper_1304_1864_gb300 as m
    cases = [_make(*r, seed=31 + i) for i, r in enumerate(REQUESTS[:4])]
    with m.Server(workers=2, hbm_budget=1) as srv:
        tickets = [srv.submit(c[0][2], c[0][3], c[0][4], c[0][5], mode=r[3], il=r[4], iu=r[5])
                   for r, c in zip(REQUESTS[:4], cases)]
        infos = [srv.poll(t) for t in tickets]
    for (rc, info), (bufs, (W1, Z1)) in zip(infos, cases):
        assert rc == 0 and info["batch"] == 1
        assert np.array_equal(_acc.as_np(bufs[4]), W1) and np.array_equal(_acc.as_np(bufs[5]).T, Z1)


def test_continuous_admission_while_busy():
    # requests keep arriving while earlier batches run; all complete, and the
    # later ones are admitted into batches of their own
    import paper_1304_1864_gb300 as m
    rng = np.random.default_rng(5)
    with m.Server(workers=2) as srv:
        tickets, bufs, infos = [], [], {}
        for i in range(24):
            n = int(rng.integers(64, 600))
            d, e = inputs.uniform_random(n, seed=100 + i)
            W = torch.empty(n, dtype=torch.float32, device="cuda")
            Z = torch.empty((n, n), dtype=torch.float32, device="cuda")
            dd = torch.tensor(d, dtype=torch.float32, device="cuda")
            ee = torch.tensor(e, dtype=torch.float32, device="cuda")
            bufs.append((d, e, W, Z))
            tickets.append(srv.submit(dd, ee, W, Z))
            if i % 6 == 5:  # wait for one request between bursts
                infos[tickets[i - 5]] = srv.poll(tickets[i - 5], wait_ms=-1)
        for t in tickets:
            if t not in infos:
                infos[t] = srv.poll(t, wait_ms=-1)
        st = srv.stats()
    assert st["completed"] == 24 and st["batches"] >= 2
    for (d, e, W, Z), t in zip(bufs, tickets):
        assert infos[t][0] == 0
        d64, e64 = _acc.exact_input(d, e, "s")
        _acc.check_res_orth(d64, e64, _acc.as_np(W).astype(np.float64), _acc.as_np(Z).T, "s", "mixed")


def test_bad_requests_are_rejected_at_submit():
    import paper_1304_1864_gb300 as m
    with m.Server() as srv:
        d = np.ones(8, np.float32)
        e = np.ones(7, np.float32)
        W = np.zeros(8, np.float32)
        Z = np.zeros((8, 8), np.float32)
        with pytest.raises(m.MrrrError):
            srv.submit(d, e, W, Z, il=3, iu=2)
        with pytest.raises(m.MrrrError):
            srv.submit(d, e, W, Z, il=1, iu=9)
        with pytest.raises(m.MrrrError):
            srv.poll(12345, wait_ms=0)


def test_cancel_withdraws_a_pending_request():
    # one worker admitting one request at a time: while a larger request
    # runs, the next one waits and can be withdrawn.  Its outputs stay as they
    # were and its poll reports MRRR_ERR_CANCELLED; the running request
    # completes as usual; a retired ticket cannot be cancelled; only completed
    # requests are counted
    import paper_1304_1864_gb300 as m
    da, ea = inputs.make("121", 2001, seed=1)
    db, eb = inputs.uniform_random(300, seed=2)
    Wa = np.full(2001, np.nan, np.float32)
    Za = np.full((2001, 2001), np.nan, np.float32)
    Wb = np.full(300, np.nan, np.float32)
    Zb = np.full((300, 300), np.nan, np.float32)
    with m.Server(workers=1, max_batch=1) as srv:
        ta = srv.submit(da.astype(np.float32), ea.astype(np.float32), Wa, Za)
        tb = srv.submit(db.astype(np.float32), eb.astype(np.float32), Wb, Zb)
        assert srv.cancel(tb) == m.MRRR_OK
        rb, _ = srv.poll(tb)
        ra, info = srv.poll(ta)
        with pytest.raises(m.MrrrError):
            srv.cancel(ta)
        st = srv.stats()
    assert rb == m.MRRR_ERR_CANCELLED and np.all(np.isnan(Wb)) and np.all(np.isnan(Zb))
    assert ra == 0 and info["m"] == 2001 and st["completed"] == 1
    d64, e64 = _acc.exact_input(da, ea, "s")
    _acc.check_res_orth(d64, e64, Wa.astype(np.float64), Za.T, "s", "mixed")


def test_out_of_memory_at_admission_fails_only_its_batch():
    # test hook (alloc_failures): the first batch fails as if its device
    # allocation had failed.  Its request completes with MRRR_ERR_NOMEM and
    # its outputs untouched; the server goes on and serves the next requests
    # as the same requests solved alone
    import paper_1304_1864_gb300 as m
    cases = [_make(*r, seed=51 + i) for i, r in enumerate(REQUESTS[1:4])]
    with m.Server(workers=1, max_batch=1, alloc_failures=1) as srv:
        tickets = [srv.submit(c[0][2], c[0][3], c[0][4], c[0][5], mode=r[3], il=r[4], iu=r[5])
                   for r, c in zip(REQUESTS[1:4], cases)]
        results = [srv.poll(t) for t in tickets]
    assert results[0][0] == m.MRRR_ERR_NOMEM and results[0][1]["m"] == 0
    assert np.all(np.isnan(_acc.as_np(cases[0][0][4])))
    for (rc, info), (bufs, (W1, Z1)) in zip(results[1:], cases[1:]):
        assert rc == 0
        assert np.array_equal(_acc.as_np(bufs[4]), W1) and np.array_equal(_acc.as_np(bufs[5]).T, Z1)
