"""Seeded synthetic test matrices (diagonal d, off-diagonal e).

This module holds no arithmetic of the eigensolver: it only draws or writes
down the entries of the test tridiagonals, and is shared by the tests, the
benchmark and the oracle checks.  The matrix types are the ones the paper
tests with (Sec. 5: uniform and geometric eigenvalue distributions, 1-2-1,
Clement, Wilkinson and Hermite matrices; glued Wilkinson matrices for tight
clusters); the paper defers their definitions to a test-matrix collection
that is not reproduced here, so each generator states the textbook
definition it uses.  The two eigenvalue-distribution types are built from a
prescribed spectrum by Lanczos (``from_spectrum``), which is a generator
step, not part of the eigensolver.

All generators return float64 arrays (d of length n, e of length n-1); a
caller that wants single-precision input casts them.
"""
import math

import numpy as np


def uniform_random(n: int, seed: int = 0):
    """d_i, e_i ~ U(-1, 1) i.i.d.: numpy PCG64 ``default_rng(seed)``, d drawn
    first (n values), then e (n-1 values)."""
    rng = np.random.default_rng(seed)
    d = rng.uniform(-1.0, 1.0, n)
    e = rng.uniform(-1.0, 1.0, max(n - 1, 0))
    return d, e


def one_two_one(n: int):
    """The 1-2-1 Toeplitz matrix: d_i = 2, e_i = -1.  Its eigenvalues are
    2 - 2 cos(k pi / (n+1)) with sine eigenvectors."""
    return np.full(n, 2.0), np.full(max(n - 1, 0), -1.0)


def wilkinson(n: int):
    """Wilkinson W_n (n = 2m+1 odd): d_i = |m + 1 - i| (1-based), e_i = 1."""
    if n % 2 != 1:
        raise ValueError("Wilkinson matrices are defined for odd n")
    m = (n - 1) // 2
    i = np.arange(1, n + 1)
    return np.abs(m + 1 - i).astype(np.float64), np.ones(n - 1)


def clement(n: int):
    """Clement matrix: d_i = 0, e_i = sqrt(i (n - i)), i = 1..n-1.  Its
    eigenvalues are the integers -(n-1), -(n-3), ..., n-1."""
    i = np.arange(1, n, dtype=np.float64)
    return np.zeros(n), np.sqrt(i * (n - i))


def hermite(n: int):
    """Jacobi matrix of the (physicists') Hermite polynomials: d_i = 0,
    e_i = sqrt(i / 2).  Its eigenvalues are the roots of H_n."""
    i = np.arange(1, n, dtype=np.float64)
    return np.zeros(n), np.sqrt(i / 2.0)


def glued_wilkinson(copies: int, block: int = 201, coupling: float = 1e-8):
    """``copies`` Wilkinson W_block matrices on the diagonal, joined by
    off-diagonal entries equal to ``coupling``."""
    db, eb = wilkinson(block)
    d = np.tile(db, copies)
    e = np.empty(copies * block - 1)
    for c in range(copies):
        e[c * block:(c + 1) * block - 1] = eb
        if c < copies - 1:
            e[(c + 1) * block - 1] = coupling
    return d, e


def glued_wilkinson_offset(copies: int, block: int, coupling: float, delta: float):
    """glued_wilkinson with block c's diagonal raised by c * delta: the
    matching eigenvalues of the copies stay close (a cluster) but apart from
    one another, so no pair is degenerate to working precision, as the
    symmetric gluing makes one."""
    d, e = glued_wilkinson(copies, block, coupling)
    return d + np.repeat(np.arange(copies) * delta, block), e


def from_spectrum(lam, seed: int = 0):
    """A symmetric tridiagonal whose eigenvalues are ``lam``: the Lanczos
    tridiagonalisation of diag(lam) from a seeded random unit start vector
    (numpy PCG64 ``default_rng(seed)``, standard normal entries), in binary64
    with full reorthogonalisation against every previous Lanczos vector,
    applied twice per step.  In exact arithmetic T has exactly the spectrum
    ``lam``; in binary64 each eigenvalue moves by O(eps ||lam||), and the
    tests take T's eigenvalues from the oracle, never from ``lam``.  Costs
    about 2 n^3 flops (a few seconds at n = 2500)."""
    lam = np.asarray(lam, np.float64)
    n = lam.size
    rng = np.random.default_rng(seed)
    Q = np.zeros((n, n))  # row j = Lanczos vector q_j
    q = rng.standard_normal(n)
    Q[0] = q / np.linalg.norm(q)
    d = np.zeros(n)
    e = np.zeros(max(n - 1, 0))
    for j in range(n):
        w = lam * Q[j]
        d[j] = Q[j] @ w
        if j == n - 1:
            break
        w -= d[j] * Q[j]
        if j > 0:
            w -= e[j - 1] * Q[j - 1]
        for _ in range(2):
            w -= Q[:j + 1].T @ (Q[:j + 1] @ w)
        b = np.linalg.norm(w)
        e[j] = b
        if b == 0.0:  # invariant subspace found: restart from a fresh direction
            w = rng.standard_normal(n)
            for _ in range(2):
                w -= Q[:j + 1].T @ (Q[:j + 1] @ w)
            b = np.linalg.norm(w)
        Q[j + 1] = w / b
    return d, e


def uniform_spectrum(n: int, seed: int = 0, eps: float = 2.0 ** -53):
    """Eigenvalues evenly spaced in [eps, 1]: lambda_i = eps + (i - 1)(1 - eps)
    / (n - 1) (the "uniform eigenvalue distribution" type of Sec. 5; the
    paper defers the definition to its test-matrix collection, this is the
    arithmetic mode of LAPACK's test-matrix generator with condition 1/eps),
    as a tridiagonal by ``from_spectrum``."""
    i = np.arange(n, dtype=np.float64)
    lam = eps + i * (1.0 - eps) / max(n - 1, 1)
    return from_spectrum(lam, seed)


def geometric_spectrum(n: int, seed: int = 0, eps: float = 2.0 ** -53):
    """Eigenvalues geometrically spaced from eps to 1: lambda_i =
    eps^((n - i) / (n - 1)) (the "geometric eigenvalue distribution" type of
    Sec. 5, the geometric mode of LAPACK's test-matrix generator with
    condition 1/eps), as a tridiagonal by ``from_spectrum``."""
    i = np.arange(1, n + 1, dtype=np.float64)
    lam = eps ** ((n - i) / max(n - 1, 1))
    return from_spectrum(lam, seed)


def make(kind: str, n: int, seed: int = 0):
    """Dispatch by type name: 'uniform' (entries U(-1, 1)), '121',
    'wilkinson', 'clement', 'hermite', 'glued' (glued copies of W_21, n
    rounded down to a multiple of 21), 'uniform_spectrum' and
    'geometric_spectrum' (the paper's two eigenvalue-distribution types)."""
    if kind == "uniform":
        return uniform_random(n, seed)
    if kind == "uniform_spectrum":
        return uniform_spectrum(n, seed)
    if kind == "geometric_spectrum":
        return geometric_spectrum(n, seed)
    if kind == "121":
        return one_two_one(n)
    if kind == "wilkinson":
        return wilkinson(n if n % 2 == 1 else n - 1)
    if kind == "clement":
        return clement(n)
    if kind == "hermite":
        return hermite(n)
    if kind == "glued":
        return glued_wilkinson(max(1, n // 21), 21, 1e-8)
    raise ValueError(kind)


# ---------------------------------------------------------------- workloads

def workload_c1():
    """Plain FP64 MRRR workload: one tridiagonal, n = 500, U(-1,1), seed 0."""
    return [uniform_random(500, 0)]


def workload_c2(n: int = 4001):
    """Mixed single/double workload: 1-2-1, Wilkinson W_n and Clement, n = 4001,
    each solved on its own (float32 input)."""
    return [one_two_one(n), wilkinson(n), clement(n)]


def workload_c3(copies: int = 40):
    """Mixed double/double-double workload: 40 glued W_201, coupling 1e-8
    (n = 8040)."""
    return [glued_wilkinson(copies, 201, 1e-8)]


BATCH_KINDS = ("uniform", "121", "wilkinson", "glued")


def workload_c4(count: int = 4096, seed: int = 4, nmin: int = 32, nmax: int = 2048):
    """Batched workload: ``count`` independent tridiagonals with n log-uniform in
    [nmin, nmax] and the type drawn uniformly from BATCH_KINDS (Wilkinson: n
    rounded down to odd; glued: copies of W_21, n rounded down to a multiple
    of 21).  Returns a list of (kind, d, e)."""
    rng = np.random.default_rng(seed)
    out = []
    for j in range(count):
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        kind = BATCH_KINDS[int(rng.integers(0, len(BATCH_KINDS)))]
        d, e = make(kind, n, seed=int(rng.integers(0, 2**31)))
        out.append((kind, d, e))
    return out


def serving_trace(rate: float = 2000.0, seconds: float = 60.0, seed: int = 5,
                  nmin: int = 64, nmax: int = 16384):
    """Poisson arrival trace for the serving loop: a list of dicts with the
    arrival time, matrix size n (log-uniform), type, input precision ('s' or
    'd', half each) and the wanted index range (all pairs, or a random
    contiguous range covering ceil(0.1 n) indices, half each)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= seconds:
            break
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        kind = BATCH_KINDS[int(rng.integers(0, len(BATCH_KINDS)))]
        prec = "s" if rng.random() < 0.5 else "d"
        if rng.random() < 0.5:
            il, iu = 1, n
        else:
            width = int(math.ceil(0.1 * n))
            il = int(rng.integers(1, n - width + 2))
            iu = il + width - 1
        out.append({"t": t, "n": n, "kind": kind, "prec": prec, "il": il, "iu": iu,
                    "seed": int(rng.integers(0, 2**31))})
    return out
