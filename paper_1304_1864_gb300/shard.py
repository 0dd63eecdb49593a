"""Index-range sharding of one tridiagonal eigenproblem over several ranks.

Every rank (one GPU each, or one process of a CPU group) holds the whole
tridiagonal.  The wanted index range 1..n is split into contiguous parts
whose boundaries lie at gaps of the root classification (mrrr_partition_s /
_d, computed redundantly and identically on every rank), each rank solves
its own part with an index-range solve, and only the results are
exchanged: an all-gather of W (n values) and, when asked for, of the column
blocks of Z.  There is no exchange during the solve.
"""
import numpy as np

from . import _binding


def _library_solver(d, e, mode, il, iu):
    W, Z, st = _binding.solve(d, e, mode=mode, range="index", il=il, iu=iu)
    return W, Z


def solve_sharded(d, e, rank, world, mode="mixed", gather="W", group=None, partitioner=None, solver=None):
    """Solve this rank's part of (d, e) and gather the results.

    d, e: the whole tridiagonal on every rank (torch tensors on this rank's
    device, or CPU tensors with a CPU process group).  gather: None (no
    exchange), "W" (every rank receives all eigenvalues) or "WZ" (also the
    full eigenvector matrix).  partitioner(d, e, world, mode) and
    solver(d, e, mode, il, iu) default to the library's partition and
    index-range solve.

    Returns a dict with 'parts' (the (il, iu) of every rank), 'W', 'Z' (this
    rank's part: W of k values, Z of n x k), and 'W_all' / 'Z_all' when
    gathered (in index order)."""
    import torch
    import torch.distributed as dist
    partitioner = partitioner or (lambda d_, e_, w_, m_: _binding.partition(d_, e_, w_, mode=m_))
    solver = solver or _library_solver
    parts = partitioner(d, e, world, mode)
    assert len(parts) == world
    il, iu = parts[rank]
    n = int(d.shape[0])
    k = iu - il + 1
    if k > 0:
        W, Z = solver(d, e, mode, il, iu)
    else:
        W = torch.empty(0, dtype=d.dtype, device=d.device)
        Z = torch.empty((n, 0), dtype=d.dtype, device=d.device)
    out = {"parts": parts, "W": W, "Z": Z}
    if not gather:
        return out
    sizes = [max(b - a + 1, 0) for a, b in parts]
    kmax = max(max(sizes), 1)
    Wp = torch.zeros(kmax, dtype=d.dtype, device=d.device)
    Wp[:k] = W
    Wg = [torch.empty_like(Wp) for _ in range(world)]
    dist.all_gather(Wg, Wp, group=group)
    out["W_all"] = torch.cat([w[:s] for w, s in zip(Wg, sizes)])
    if gather == "WZ":
        # column blocks, sent as rows of the transposed (k x n) block
        Zp = torch.zeros((kmax, n), dtype=d.dtype, device=d.device)
        Zp[:k] = Z.T
        Zg = [torch.empty_like(Zp) for _ in range(world)]
        dist.all_gather(Zg, Zp, group=group)
        out["Z_all"] = torch.cat([z[:s] for z, s in zip(Zg, sizes)]).T
    return out


def even_parts(n, world):
    """The even split of 1..n into `world` contiguous ranges (the partition
    of a matrix without usable gaps, and a stand-in partitioner for tests)."""
    cut = [int((n * p + world // 2) // world) for p in range(world + 1)]
    return [(cut[p] + 1, cut[p + 1]) for p in range(world)]


def check_parts(parts, n):
    """The parts tile 1..n in order (empty parts allowed)."""
    nxt = 1
    for a, b in parts:
        if a != nxt or b < a - 1:
            return False
        nxt = b + 1
    return nxt == n + 1 and bool(np.all([b >= a - 1 for a, b in parts]))
