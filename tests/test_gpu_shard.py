"""The index-range split for independent solves (one part per GPU): the
partition boundaries lie at gaps of the root classification, and the parts
solved one by one (here in turn on one GPU, as the ranks of a multi-GPU run
would solve them at once) give together every eigenpair of the matrix, each
eigenvalue within the oracle tolerance and the union of the vectors
orthogonal to the method's target."""
import numpy as np
import pytest

from paper_1304_1864_gb300 import inputs

from . import _acc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _parts_union(d, e, prec, nparts):
    import paper_1304_1864_gb300 as m
    from paper_1304_1864_gb300 import shard
    dt = torch.float32 if prec == "s" else torch.float64
    dg = torch.tensor(np.asarray(d), dtype=dt, device="cuda")
    eg = torch.tensor(np.asarray(e), dtype=dt, device="cuda")
    n = dg.shape[0]
    parts = m.partition(dg, eg, nparts, mode="mixed")
    assert shard.check_parts(parts, n), parts
    Ws, Zs = [], []
    for il, iu in parts:
        if il > iu:
            continue
        W, Z, st = m.solve(dg, eg, mode="mixed", range="index", il=il, iu=iu)
        assert st["status"] == 0 and W.shape[0] == iu - il + 1
        Ws.append(_acc.as_np(W))
        Zs.append(_acc.as_np(Z))
    torch.cuda.synchronize()
    return parts, np.concatenate(Ws), np.concatenate(Zs, axis=1)


@pytest.mark.parametrize("nparts", [2, 4, 8])
@pytest.mark.parametrize("which", [0, 1, 2], ids=["121", "wilkinson", "clement"])
def test_sharded_n4001_fp32(which, nparts):
    names = ("121", "wilkinson", "clement")
    d, e = inputs.workload_c2()[which]
    d64, e64 = _acc.exact_input(d, e, "s")
    parts, W, Z = _parts_union(d, e, "s", nparts)
    # the boundaries move off the even split only as far as the nearest gap
    assert sum(1 for a, b in parts if a <= b) >= nparts - 1
    assert np.all(np.diff(W) >= 0)
    _acc.check_eigvals_all(d64, e64, W, "s", "mixed", _acc.oracle_all("c2-" + names[which], d64, e64))
    _acc.check_res_orth(d64, e64, W, Z, "s", "mixed")


def test_sharded_glued_wilkinson_fp64():
    # tight clusters of 80: boundaries must not cut them
    d, e = inputs.workload_c3()[0]
    parts, W, Z = _parts_union(d, e, "d", 4)
    _acc.check_eigvals_all(d, e, W, "d", "mixed", _acc.oracle_all("c3", d, e))
    _acc.check_res_orth(d, e, W, Z, "d", "mixed")


def test_sharded_split_matrix_even_parts():
    # a matrix that splits into blocks is cut evenly (blocks are independent)
    d, e = inputs.glued_wilkinson(6, 21, 1e-20)
    d64, e64 = _acc.exact_input(d, e, "d")
    parts, W, Z = _parts_union(d, e, "d", 3)
    assert parts == [(1, 42), (43, 84), (85, 126)]
    _acc.check_eigvals(d64, e64, W, "d", "mixed")
    _acc.check_res_orth(d64, e64, W, Z, "d", "mixed")


def test_partition_arguments():
    import paper_1304_1864_gb300 as m
    d = torch.ones(10, dtype=torch.float64, device="cuda")
    e = torch.full((9,), 0.5, dtype=torch.float64, device="cuda")
    assert m.partition(d, e, 1) == [(1, 10)]
    with pytest.raises(m.MrrrError):
        m.partition(d, e, 0)
    parts = m.partition(d[:2], e[:1], 4)
    assert len(parts) == 4 and sum(max(b - a + 1, 0) for a, b in parts) == 2
