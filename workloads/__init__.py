"""Seeded synthetic inputs shaped like the paper's least-squares workloads.

This module is shared by the tests, the benchmark and the oracle checks; it
holds no arithmetic of the factorization itself, only random-number draws
(numpy ``default_rng``) and, for the conditioned matrices, a library QR
(LAPACK through numpy) used to draw random orthogonal factors.

All matrices are returned column-major (Fortran order), FP64.

Recipes (the paper states neither the matrix contents nor the precision of its
runs; its experiments use dense square matrices, Section 4.2):

* ``gaussian(m, n, seed)``      iid N(0,1) entries; RHS iid N(0,1).
* ``conditioned(m, n, kappa)``  U diag(sigma) V^T with U, V random orthogonal
  and sigma_i = kappa^(-i/(n-1)); consistent RHS b = A x_true and N(0,1) RHS.
* ``batch_shapes(count)``       m ~ U{16..512}, n ~ U{ceil(m/4)..m}.
* ``slsqp_stack(n, m_eq)``      the stacked SLSQP LS matrix [L^T; C], L lower
  triangular with diagonal ~ U[0.5, 2] and N(0, 0.1) strictly-lower entries,
  C ~ N(0,1).
"""
from __future__ import annotations

import math

import numpy as np

# Seeds per workload: one fixed seed per configuration so that every run of the
# tests, the benchmark and the oracle sees identical bytes.
SEED_SMALL = 1          # 256 x 128
SEED_TALL = 2           # 16384 x 2048
SEED_SQUARE = 3         # 8192 x 8192
SEED_COND = {1e2: 4, 1e6: 5, 1e10: 6}   # 8192 x 4096 conditioned
SEED_BATCH = 7          # 20,000 uneven problems
SEED_SERVE = 8          # request stream


def gaussian(m: int, n: int, seed: int):
    """(A, b): A m x n iid N(0,1) (column-major), b length m iid N(0,1)."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal(size=(n, m)).T  # Fortran-ordered m x n
    b = rng.standard_normal(size=m)
    return A, b


def gaussian_rhs(m: int, nrhs: int, seed: int):
    """An m x nrhs block of iid N(0,1) right-hand sides (column-major)."""
    rng = np.random.default_rng(seed + 1000)
    return rng.standard_normal(size=(nrhs, m)).T


def _random_orthogonal(rows: int, cols: int, rng) -> np.ndarray:
    """Columns of a random orthogonal factor: Q of a Gaussian matrix, with the
    column signs fixed so that diag(R) > 0 (library QR, LAPACK)."""
    G = rng.standard_normal(size=(rows, cols))
    Q, R = np.linalg.qr(G)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s


def conditioned(m: int, n: int, kappa: float, seed: int | None = None):
    """(A, b_consistent, x_true, b_random) with cond_2(A) = kappa.

    A = U diag(sigma) V^T, sigma_i = kappa^(-i/(n-1)), i = 0..n-1.
    """
    if seed is None:
        seed = SEED_COND.get(kappa, 4)
    rng = np.random.default_rng(seed)
    U = _random_orthogonal(m, n, rng)
    V = _random_orthogonal(n, n, rng)
    if n > 1:
        sigma = kappa ** (-np.arange(n) / (n - 1))
    else:
        sigma = np.ones(1)
    A = np.asfortranarray((U * sigma) @ V.T)
    x_true = rng.standard_normal(size=n)
    b_cons = A @ x_true
    b_rand = rng.standard_normal(size=m)
    return A, b_cons, x_true, b_rand


def conditioned_device(m: int, n: int, kappa: float, seed: int | None = None, device="cuda"):
    """The `conditioned` recipe drawn on the device (torch RNG, library QR):
    (A, b_consistent, x_true, b_random) as column-major float64 CUDA tensors."""
    import torch
    if seed is None:
        seed = SEED_COND.get(kappa, 4)
    g = torch.Generator(device=device)
    g.manual_seed(seed)

    def orth(rows, cols):
        Gm = torch.randn(rows, cols, generator=g, dtype=torch.float64, device=device)
        Q, R = torch.linalg.qr(Gm)
        sgn = torch.sign(torch.diagonal(R))
        sgn[sgn == 0] = 1.0
        return Q * sgn

    U = orth(m, n)
    V = orth(n, n)
    if n > 1:
        sigma = kappa ** (-torch.arange(n, dtype=torch.float64, device=device) / (n - 1))
    else:
        sigma = torch.ones(1, dtype=torch.float64, device=device)
    A = (U * sigma) @ V.T
    A = A.t().contiguous().t()                      # column-major
    x_true = torch.randn(n, generator=g, dtype=torch.float64, device=device)
    b_cons = A @ x_true
    b_rand = torch.randn(m, generator=g, dtype=torch.float64, device=device)
    return A, b_cons, x_true, b_rand


def batch_shapes(count: int, seed: int = SEED_BATCH, m_lo: int = 16, m_hi: int = 512):
    """Shapes of ``count`` independent problems: m ~ U{m_lo..m_hi},
    n ~ U{ceil(m/4)..m}."""
    rng = np.random.default_rng(seed)
    ms = rng.integers(m_lo, m_hi + 1, size=count)
    ns = np.array([rng.integers(int(math.ceil(m / 4)), m + 1) for m in ms])
    return ms.astype(np.int64), ns.astype(np.int64)


def batch_problems(ms, ns, seed: int = SEED_BATCH):
    """One (A, b) per shape, iid N(0,1), each A column-major."""
    rng = np.random.default_rng(seed + 1)
    out = []
    for m, n in zip(ms, ns):
        A = rng.standard_normal(size=(int(n), int(m))).T
        b = rng.standard_normal(size=int(m))
        out.append((A, b))
    return out


def batch_problems_device(ms, ns, seed: int = SEED_BATCH, device="cuda", with_rhs=True):
    """All problems of a batch drawn on the device in one seeded stream.

    Returns (A_flat, b_flat, a_off, b_off): problem i is the column-major
    m_i x n_i block A_flat[a_off[i] : a_off[i] + m_i*n_i] (lda = m_i) and its
    right-hand side b_flat[b_off[i] : b_off[i] + m_i]; entries iid N(0,1).
    """
    import torch
    ms = [int(m) for m in ms]
    ns = [int(n) for n in ns]
    a_sizes = np.array([m * n for m, n in zip(ms, ns)], dtype=np.int64)
    b_sizes = np.array(ms, dtype=np.int64)
    a_off = np.concatenate([[0], np.cumsum(a_sizes)[:-1]]) if len(ms) else np.zeros(0, np.int64)
    b_off = np.concatenate([[0], np.cumsum(b_sizes)[:-1]]) if len(ms) else np.zeros(0, np.int64)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    A_flat = torch.randn(int(a_sizes.sum()) + 1, generator=g, dtype=torch.float64, device=device)
    b_flat = torch.randn(int(b_sizes.sum()) + 1, generator=g, dtype=torch.float64, device=device)
    return A_flat, b_flat, a_off, b_off


def slsqp_stack(n: int, m_eq: int, seed: int):
    """(A, b): A = [L^T; C] of shape (n + m_eq) x n, b ~ N(0,1).

    L is lower triangular with diagonal ~ U[0.5, 2] and strictly-lower entries
    ~ N(0, 0.1) (standard deviation 0.1); C is an m_eq x n N(0,1) block.
    """
    rng = np.random.default_rng(seed)
    L = np.tril(rng.normal(0.0, 0.1, size=(n, n)), -1)
    L[np.diag_indices(n)] = rng.uniform(0.5, 2.0, size=n)
    C = rng.standard_normal(size=(m_eq, n))
    A = np.asfortranarray(np.vstack([L.T, C]))
    b = rng.standard_normal(size=n + m_eq)
    return A, b


def serving_stream(count: int, rate: float, seed: int = SEED_SERVE,
                   n_lo: int = 50, n_hi: int = 2000):
    """Arrival times (s) and shapes of a Poisson request stream.

    n ~ log-uniform on [n_lo, n_hi], m_eq ~ U{0..floor(n/2)}; inter-arrival
    times ~ Exp(rate).  Returns (t_arrival, n, m_eq, seeds).
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps) - gaps[0]
    n = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count)).astype(np.int64)
    n = np.clip(n, n_lo, n_hi)
    m_eq = np.array([rng.integers(0, k // 2 + 1) for k in n], dtype=np.int64)
    seeds = rng.integers(0, 2**31 - 1, size=count)
    return t, n, m_eq, seeds
