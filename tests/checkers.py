"""Independent checkers used by the tests (plain torch, any device).

They rebuild the action of Q = H_0 H_1 ... H_{K-1} from a factorization in H12
storage (F, up) with the textbook compact-WY recurrence for T (LAPACK larft
style: T[:j, j] = -tau_j T[:j,:j] V[:, :j]^T v_j), independently of both the
oracle (sequential reflectors) and the CUDA path (UT-form forward
substitution).  They are pinned against the oracle in tests/test_checkers.py.
"""
from __future__ import annotations

import torch


def num_reflectors(m: int, n: int) -> int:
    return max(0, min(m - 1, n))


def _block(F, up, k0, k1):
    m = F.shape[0]
    nb = k1 - k0
    V = torch.tril(F[k0:, k0:k1], -1).clone()
    idx = torch.arange(nb, device=F.device)
    V[idx, idx] = up[k0:k1]
    b = up[k0:k1] * torch.diagonal(F[k0:k1, k0:k1])
    tau = torch.where(b < 0, -1.0 / torch.where(b < 0, b, torch.ones_like(b)),
                      torch.zeros_like(b))
    V = V * (tau != 0).to(V.dtype)            # a skipped reflector is the identity
    G = V.T @ V
    T = torch.zeros(nb, nb, dtype=F.dtype, device=F.device)
    for j in range(nb):
        if j:
            T[:j, j] = -tau[j] * (T[:j, :j] @ G[:j, j])
        T[j, j] = tau[j]
    return V, T


def apply_qt(F, up, X, nb: int = 64):
    """Q^T X (X is m x r; a copy is returned)."""
    X = X.clone()
    m, n = F.shape
    K = num_reflectors(m, n)
    for k0 in range(0, K, nb):
        k1 = min(K, k0 + nb)
        V, T = _block(F, up, k0, k1)
        X[k0:] -= V @ (T.T @ (V.T @ X[k0:]))
    return X


def apply_q(F, up, X, nb: int = 64):
    """Q X (X is m x r; a copy is returned)."""
    X = X.clone()
    m, n = F.shape
    K = num_reflectors(m, n)
    starts = list(range(0, K, nb))
    for k0 in reversed(starts):
        k1 = min(K, k0 + nb)
        V, T = _block(F, up, k0, k1)
        X[k0:] -= V @ (T @ (V.T @ X[k0:]))
    return X


def backward_error_estimate(A0, F, up, probes: int = 16, seed: int = 0):
    """||A0 - Q R||_F / ||A0||_F estimated with Gaussian probes Z (n x probes):
    E ||E Z||_F^2 = probes ||E||_F^2."""
    m, n = A0.shape
    g = torch.Generator(device="cpu").manual_seed(seed)
    Z = torch.randn(n, probes, generator=g, dtype=A0.dtype).to(A0.device)
    R = torch.triu(F[:n, :n])
    RZ = torch.zeros(m, probes, dtype=A0.dtype, device=A0.device)
    RZ[:n] = R @ Z
    E = A0 @ Z - apply_q(F, up, RZ)
    return float(torch.linalg.norm(E) / (probes ** 0.5) / torch.linalg.norm(A0))


def cond_estimate(R, iters: int = 40, seed: int = 0):
    """kappa_2(R) by power iteration on R^T R and inverse iteration with two
    triangular solves (R is square upper triangular, nonsingular)."""
    n = R.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    v = torch.randn(n, 1, generator=g, dtype=R.dtype).to(R.device)
    w = v.clone()
    smax = smin_inv = 0.0
    for _ in range(iters):
        v = R.T @ (R @ v)
        smax = float(torch.linalg.norm(v)) ** 0.5
        v = v / torch.linalg.norm(v)
        y = torch.linalg.solve_triangular(R.T, w, upper=False)
        w = torch.linalg.solve_triangular(R, y, upper=True)
        smin_inv = float(torch.linalg.norm(w)) ** 0.5
        w = w / torch.linalg.norm(w)
    return smax * smin_inv


def norm2_estimate(R, iters: int = 40, seed: int = 1):
    """||R||_2 by power iteration on R^T R."""
    n = R.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    v = torch.randn(n, 1, generator=g, dtype=R.dtype).to(R.device)
    s = 0.0
    for _ in range(iters):
        v = R.T @ (R @ v)
        s = float(torch.linalg.norm(v)) ** 0.5
        v = v / torch.linalg.norm(v)
    return s
