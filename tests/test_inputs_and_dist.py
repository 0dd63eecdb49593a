"""CPU checks of the synthetic input generators and of the multi-rank timing
helper of bench.py (two gloo ranks)."""
import math
import os
import socket

import numpy as np
import pytest

from paper_1304_1864_gb300 import inputs


def test_generators_follow_their_definitions():
    d, e = inputs.wilkinson(7)
    assert list(d) == [3, 2, 1, 0, 1, 2, 3] and np.all(e == 1)
    d, e = inputs.clement(5)
    assert np.all(d == 0) and np.allclose(e, np.sqrt([4, 6, 6, 4]))
    d, e = inputs.one_two_one(4)
    assert np.all(d == 2) and np.all(e == -1)
    d, e = inputs.hermite(4)
    assert np.allclose(e, np.sqrt([0.5, 1.0, 1.5]))
    d, e = inputs.glued_wilkinson(3, 5, 1e-8)
    assert d.size == 15 and e[4] == 1e-8 and e[9] == 1e-8 and e[3] == 1
    with pytest.raises(ValueError):
        inputs.wilkinson(4)


def test_uniform_is_seeded_and_reproducible():
    a = inputs.uniform_random(100, 0)
    b = inputs.uniform_random(100, 0)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    rng = np.random.default_rng(0)
    assert np.array_equal(a[0], rng.uniform(-1, 1, 100))
    assert np.all(np.abs(a[0]) <= 1) and a[1].size == 99


def test_workload_shapes():
    c2 = inputs.workload_c2()
    assert [d.size for d, _ in c2] == [4001, 4001, 4001]
    (d3, e3), = inputs.workload_c3()
    assert d3.size == 8040 and np.sum(e3 == 1e-8) == 39
    batch = inputs.workload_c4(count=64)
    ns = [d.size for _, d, _ in batch]
    assert len(batch) == 64 and min(ns) >= 20 and max(ns) <= 2048
    assert {k for k, _, _ in batch} <= set(inputs.BATCH_KINDS)


def test_serving_trace():
    tr = inputs.serving_trace(rate=200.0, seconds=2.0, seed=5)
    assert 300 < len(tr) < 500
    ts = [r["t"] for r in tr]
    assert ts == sorted(ts) and ts[-1] < 2.0
    for r in tr:
        assert 64 <= r["n"] <= 16384 and 1 <= r["il"] <= r["iu"] <= r["n"]
        if r["iu"] - r["il"] + 1 != r["n"]:
            assert r["iu"] - r["il"] + 1 == math.ceil(0.1 * r["n"])


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    v = bench._max_over_ranks(float(rank + 1) * 10.0, world)
    bench._barrier(world)
    q.put((rank, v))
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    q = ctx.Queue()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(out) == [(0, 20.0), (1, 20.0)]


@pytest.mark.parametrize("kind", ["uniform_spectrum", "geometric_spectrum"])
def test_spectrum_generators_reach_their_spectrum(kind):
    # the Lanczos tridiagonal of diag(lambda) has the prescribed eigenvalues up
    # to binary64 rounding (LAPACK's tridiagonal eigenvalues as the check)
    sl = pytest.importorskip("scipy.linalg")
    n = 300
    d, e = inputs.make(kind, n, seed=3)
    lam = sl.eigvalsh_tridiagonal(d, e)
    i = np.arange(n)
    eps = 2.0 ** -53
    want = eps + i * (1 - eps) / (n - 1) if kind == "uniform_spectrum" else eps ** ((n - 1 - i) / (n - 1))
    assert np.max(np.abs(lam - want)) <= 64 * n * eps
    # seeded: the same matrix every time, another one for another seed
    d2, e2 = inputs.make(kind, n, seed=3)
    assert np.array_equal(d, d2) and np.array_equal(e, e2)
    d3, _ = inputs.make(kind, n, seed=4)
    assert not np.array_equal(d, d3)


def _cpu_part_solver(d, e, mode, il, iu):
    # stand-in for the GPU solve of an index range (LAPACK, binary64), so that
    # the sharding logic runs without a GPU
    import torch
    sl = pytest.importorskip("scipy.linalg")
    w, v = sl.eigh_tridiagonal(d.numpy(), e.numpy(), select="i", select_range=(il - 1, iu - 1))
    return torch.from_numpy(w), torch.from_numpy(np.ascontiguousarray(v))


def _shard_worker(rank, world, port, parts, q):
    import torch
    import torch.distributed as dist
    from paper_1304_1864_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    d, e = inputs.uniform_random(60, 9)
    out = shard.solve_sharded(torch.from_numpy(d), torch.from_numpy(e), rank, world, gather="WZ",
                              partitioner=lambda d_, e_, w_, m_: parts, solver=_cpu_part_solver)
    q.put((rank, out["W"].numpy(), out["W_all"].numpy(), out["Z_all"].numpy()))
    dist.destroy_process_group()


@pytest.mark.parametrize("parts", [[(1, 25), (26, 60)], [(1, 60), (61, 60)], [(1, 0), (1, 60)]],
                         ids=["uneven", "empty-last", "empty-first"])
def test_sharded_solve_gathers_two_gloo_ranks(parts):
    # two CPU ranks, each solving its index range; the all-gathered W and Z
    # are the parts in index order, identical on both ranks
    import multiprocessing as mp
    from paper_1304_1864_gb300 import shard
    assert shard.check_parts(parts, 60)
    ctx = mp.get_context("spawn")
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    q = ctx.Queue()
    ps = [ctx.Process(target=_shard_worker, args=(r, 2, port, parts, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    torch = pytest.importorskip("torch")
    d, e = inputs.uniform_random(60, 9)
    want_w, want_z = [], []
    for a, b in parts:
        if a <= b:
            w, z = _cpu_part_solver(torch.from_numpy(d), torch.from_numpy(e), "mixed", a, b)
            want_w.append(w.numpy())
            want_z.append(z.numpy())
    want_w = np.concatenate(want_w)
    want_z = np.concatenate(want_z, axis=1)
    for rank, w_own, w_all, z_all in out:
        a, b = parts[rank]
        assert w_own.size == max(b - a + 1, 0)
        assert np.array_equal(w_all, want_w) and np.array_equal(z_all, want_z)


def test_partition_helpers():
    from paper_1304_1864_gb300 import shard
    for n, world in [(10, 3), (1, 4), (0, 2), (4001, 8)]:
        parts = shard.even_parts(n, world)
        assert len(parts) == world and shard.check_parts(parts, n)
    assert not shard.check_parts([(1, 5), (7, 10)], 10)
    assert not shard.check_parts([(1, 5), (6, 9)], 10)


@pytest.mark.parametrize("prec,coupling,delta", [("d", 1e-8, 1e-6), ("s", 1.5e-6, 1e-4)])
def test_offset_glued_wilkinson_nests_clusters_without_a_degenerate_pair(prec, coupling, delta):
    # the input of the backtracking test, from the oracle's eigenvalues: the
    # top 24 eigenvalues lie within 1e-3 of one another relative to their
    # size (one cluster at the root for gaptol 1e-3); they come in pairs much
    # closer than the spread of the set (each pair a cluster again in the
    # child made for the set) with the pairs well apart; and no two
    # eigenvalues of the matrix agree to binary64 resolution.  The plain
    # gluing of the same blocks has a pair that does.
    import oracle

    def eig(d, e):
        if prec == "s":
            d, e = d.astype(np.float32).astype(np.float64), e.astype(np.float32).astype(np.float64)
        hi, lo = oracle.eigvals(d, e)
        return hi, lo

    hi, lo = eig(*inputs.glued_wilkinson_offset(12, 21, coupling, delta))
    th, tl = hi[-24:], lo[-24:]
    spread = (th[-1] - th[0]) + (tl[-1] - tl[0])
    assert spread < 1e-3 * abs(th[0])
    gaps = np.diff(th) + np.diff(tl)
    assert np.all(gaps[0::2] < 1e-3 * spread / 4) and np.all(gaps[1::2] > 1e-3 * spread)
    eps_d = 2.0 ** -53
    assert (np.diff(hi) + np.diff(lo)).min() > 1e3 * eps_d * np.abs(hi).max()
    h0, l0 = eig(*inputs.glued_wilkinson(12, 21, coupling))
    assert (np.diff(h0) + np.diff(l0)).min() < eps_d * np.abs(h0).max()
