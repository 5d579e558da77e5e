"""CPU oracle for the H12 Householder QR, Q^T.B application and back-substitution.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import this package.  The product path
(``paper_2506_09463_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``h12_oracle.c`` (plain sequential C, binary64, no BLAS),
which follows Alg. 2 of the paper (Section 3) with the two kernels
``update_pivot_row`` / ``update_trailing_non_pivot_row`` and the Task 1 skip rule
(Alg. 3), in the Lawson-Hanson H12 storage form.  This module compiles it with
gcc on first use and wraps it with ctypes over numpy arrays.

Every function here is pinned by the CPU tests (``tests/test_oracle_*.py``)
against hand-worked exact examples, exact rational normal equations, invariants
of Alg. 1 and special cases.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "h12_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle_h12.so")
_lock = threading.Lock()
_lib = None

ERANK = -5


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle_h12.so`` (gcc -O2)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            i = ctypes.c_int
            lib.oracle_num_reflectors.argtypes = [i, i]
            lib.oracle_num_reflectors.restype = i
            lib.oracle_h12_factor.argtypes = [i, i, dp, i, dp]
            lib.oracle_h12_factor.restype = i
            lib.oracle_apply_qt.argtypes = [i, i, dp, i, dp, i, dp, i]
            lib.oracle_apply_qt.restype = None
            lib.oracle_apply_q.argtypes = [i, i, dp, i, dp, i, dp, i]
            lib.oracle_apply_q.restype = None
            lib.oracle_solve_r.argtypes = [i, dp, i, i, dp, i]
            lib.oracle_solve_r.restype = i
            lib.oracle_residual_norm.argtypes = [i, i, dp]
            lib.oracle_residual_norm.restype = ctypes.c_double
            lib.oracle_lstsq.argtypes = [i, i, dp, i, dp, dp]
            lib.oracle_lstsq.restype = i
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _colmajor(a) -> np.ndarray:
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        a = a.reshape(-1, 1)
    return np.asfortranarray(a)


def num_reflectors(m: int, n: int) -> int:
    """min(m-1, n): a length-1 vector gets no reflector."""
    return _load().oracle_num_reflectors(m, n)


def h12_factor(A):
    """Factor a copy of ``A`` (m x n).  Returns ``(F, up, skipped)``.

    ``F`` holds R in its upper triangle and the reflector tails below the
    diagonal (column-major, ``F[k,k] = R_kk``); ``up[k]`` is the pivot entry of
    reflector k (0 for skipped pivots and for k >= min(m-1, n)).
    """
    F = _colmajor(A).copy(order="F")
    m, n = F.shape
    up = np.zeros(n, dtype=np.float64)
    if m == 0 or n == 0:
        return F, up, 0
    skipped = _load().oracle_h12_factor(m, n, _ptr(F), m, _ptr(up))
    return F, up, skipped


def apply_qt(F, up, B):
    """Return Q^T B for the factorization ``(F, up)``; B is m x nrhs (or m)."""
    F = _colmajor(F)
    vec = np.asarray(B).ndim == 1
    Bc = _colmajor(B).copy(order="F")
    m, n = F.shape
    up = np.ascontiguousarray(up, dtype=np.float64)
    if m and Bc.shape[1]:
        _load().oracle_apply_qt(m, n, _ptr(F), m, _ptr(up), Bc.shape[1], _ptr(Bc), m)
    return Bc[:, 0].copy() if vec else Bc


def apply_q(F, up, B):
    """Return Q B = H_0 H_1 ... H_{K-1} B for the factorization ``(F, up)``."""
    F = _colmajor(F)
    vec = np.asarray(B).ndim == 1
    Bc = _colmajor(B).copy(order="F")
    m, n = F.shape
    up = np.ascontiguousarray(up, dtype=np.float64)
    if m and Bc.shape[1]:
        _load().oracle_apply_q(m, n, _ptr(F), m, _ptr(up), Bc.shape[1], _ptr(Bc), m)
    return Bc[:, 0].copy() if vec else Bc


def solve_r(F, C):
    """Back-substitute R X = C[0:n] (R = triu(F[0:n,0:n])).  Returns ``(X, status)``.

    ``C`` has at least n rows; only its first n rows are used.  status is 0 or
    ERANK (-5) when some R_ii == 0 (that unknown is set to 0).
    """
    F = _colmajor(F)
    n = F.shape[1]
    vec = np.asarray(C).ndim == 1
    Cc = _colmajor(C)[:n].copy(order="F")
    status = 0
    if n and Cc.shape[1]:
        status = _load().oracle_solve_r(n, _ptr(F), F.shape[0], Cc.shape[1], _ptr(Cc), n)
    return (Cc[:, 0].copy() if vec else Cc), status


def residual_norm(qtb, n: int) -> float:
    """||(Q^T b)[n:m]||_2 for one right-hand side (the LS residual norm)."""
    q = np.ascontiguousarray(qtb, dtype=np.float64).ravel()
    return float(_load().oracle_residual_norm(q.shape[0], n, _ptr(q)))


def lstsq(A, b):
    """Full LS solve of one problem: factor, Q^T b, back-substitute.

    Returns ``(x, F, up, qtb, status)``.
    """
    F, up, _ = h12_factor(A)
    qtb = apply_qt(F, up, np.asarray(b, dtype=np.float64))
    x, status = solve_r(F, qtb)
    return x, F, up, qtb, status


def r_factor(F) -> np.ndarray:
    """R as a dense n x n upper-triangular array taken from the stored form."""
    F = np.asarray(F)
    n = F.shape[1]
    return np.triu(F[:n, :n])


def reflector_vectors(F, up) -> np.ndarray:
    """The unnormalised reflector vectors v_k = (0.., up_k, F[k+1:m, k]) as columns."""
    F = np.asarray(F)
    m, n = F.shape
    K = num_reflectors(m, n)
    V = np.zeros((m, K))
    for k in range(K):
        V[k, k] = up[k]
        V[k + 1:, k] = F[k + 1:, k]
    return V
