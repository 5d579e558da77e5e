"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* hand-worked exact examples (tests/golden/), each also checked against the
  exact normal equations A^T A x = A^T b in rational arithmetic;
* brute-force exact rational least squares on tiny integer problems;
* invariants of Alg. 1 (Section 2.2): A = Q R, Q^T Q = I, R upper triangular,
  column norms preserved, v^T v = -2 b for every H12 reflector;
* special cases with closed forms (upper-triangular input, orthogonal input,
  zero column, x0 = 0, a single column, over/underflow-safe norms);
* library cross-checks (LAPACK through numpy/scipy), run as checkers only.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads

U = 2.0 ** -53
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# helpers (exact arithmetic, no oracle code)
# ----------------------------------------------------------------------------
def load_golden(name):
    rows = {"A": [], "F": []}
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *items = line.split()
            fr = [Fraction(x) for x in items]
            if key in rows:
                rows[key].append(fr)
            else:
                vals[key] = fr
    vals["A"] = rows["A"]
    vals["F"] = rows["F"]
    return vals


def exact_normal_equations(A, b):
    """Solve A^T A x = A^T b exactly (Gauss-Jordan over the rationals)."""
    m, n = len(A), len(A[0])
    M = [[sum(A[k][i] * A[k][j] for k in range(m)) for j in range(n)] +
         [sum(A[k][i] * b[k] for k in range(m))] for i in range(n)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        piv = M[c][c]
        M[c] = [v / piv for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [a - f * bb for a, bb in zip(M[r], M[c])]
    return [M[i][n] for i in range(n)]


def exact_rank(A):
    M = [list(map(Fraction, r)) for r in A]
    m, n = len(M), len(M[0])
    rank = 0
    for c in range(n):
        p = next((r for r in range(rank, m) if M[r][c] != 0), None)
        if p is None:
            continue
        M[rank], M[p] = M[p], M[rank]
        for r in range(rank + 1, m):
            f = M[r][c] / M[rank][c]
            M[r] = [a - f * bb for a, bb in zip(M[r], M[rank])]
        rank += 1
    return rank


def close(actual, expected, ulps=8):
    expected = np.asarray(expected, dtype=np.float64)
    scale = max(1.0, float(np.max(np.abs(expected)))) if expected.size else 1.0
    np.testing.assert_allclose(actual, expected, rtol=0, atol=ulps * U * scale)


def q_explicit(F, up):
    m = F.shape[0]
    return oracle.apply_q(F, up, np.eye(m))


def r_full(F):
    m, n = F.shape
    R = np.zeros((m, n))
    R[:n, :n] = np.triu(F[:n, :n])
    if m < n:
        raise ValueError
    return R


# ----------------------------------------------------------------------------
# hand-worked examples
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["h12_3x2.txt", "h12_4x3.txt"])
def test_golden_example(name):
    g = load_golden(name)
    A = np.array([[float(v) for v in r] for r in g["A"]])
    b = np.array([float(v) for v in g["b"]])
    F, up, skipped = oracle.h12_factor(A)
    assert skipped == 0
    close(F, [[float(v) for v in r] for r in g["F"]])
    close(up, [float(v) for v in g["up"]])
    qtb = oracle.apply_qt(F, up, b)
    close(qtb, [float(v) for v in g["qtb"]])
    x, status = oracle.solve_r(F, qtb)
    assert status == 0
    close(x, [float(v) for v in g["x"]])
    n = A.shape[1]
    res = oracle.residual_norm(qtb, n)
    close(res * res, float(g["res2"][0]), ulps=32)


@pytest.mark.parametrize("name", ["h12_3x2.txt", "h12_4x3.txt"])
def test_golden_solution_is_the_exact_least_squares_solution(name):
    """The golden x is pinned by the exact normal equations, independently of
    the hand derivation; the golden residual by ||b - A x||^2 exactly."""
    g = load_golden(name)
    x = exact_normal_equations(g["A"], g["b"])
    assert x == g["x"]
    r = [bi - sum(a * xi for a, xi in zip(row, x)) for row, bi in zip(g["A"], g["b"])]
    assert sum(v * v for v in r) == g["res2"][0]


def test_golden_r_matches_exact_gram():
    """R^T R = A^T A exactly for the golden R (rational arithmetic)."""
    for name in ["h12_3x2.txt", "h12_4x3.txt"]:
        g = load_golden(name)
        A, F = g["A"], g["F"]
        n = len(A[0])
        R = [[F[i][j] if j >= i else Fraction(0) for j in range(n)] for i in range(n)]
        for i in range(n):
            for j in range(n):
                ata = sum(A[k][i] * A[k][j] for k in range(len(A)))
                rtr = sum(R[k][i] * R[k][j] for k in range(n))
                assert ata == rtr


# ----------------------------------------------------------------------------
# brute force on tiny inputs
# ----------------------------------------------------------------------------
def test_bruteforce_exact_least_squares_small_integer():
    rng = np.random.default_rng(12345)
    checked = 0
    while checked < 60:
        n = int(rng.integers(1, 6))
        m = int(rng.integers(n, 9))
        Ai = rng.integers(-5, 6, size=(m, n))
        bi = rng.integers(-5, 6, size=m)
        A = [[Fraction(int(v)) for v in r] for r in Ai]
        if exact_rank(A) < n:
            continue
        xe = np.array([float(v) for v in exact_normal_equations(A, [Fraction(int(v)) for v in bi])])
        x, F, up, qtb, status = oracle.lstsq(Ai.astype(float), bi.astype(float))
        assert status == 0
        kappa = np.linalg.cond(Ai.astype(float))
        err = np.linalg.norm(x - xe) / max(np.linalg.norm(xe), 1e-300)
        # for the integer examples b may be far from range(A): LS bound
        bound = 1e3 * (kappa + kappa ** 2) * 2.0 ** -52
        assert err <= bound, (m, n, err, bound)
        checked += 1


# ----------------------------------------------------------------------------
# invariants of Alg. 1 on random inputs
# ----------------------------------------------------------------------------
SHAPES = [(1, 1), (2, 1), (2, 2), (3, 3), (5, 5), (17, 3), (33, 33), (64, 40), (100, 7),
          (129, 65)]


@pytest.mark.parametrize("m,n", SHAPES)
def test_invariants(m, n):
    A, _ = workloads.gaussian(m, n, seed=100 + m * 7 + n)
    F, up, skipped = oracle.h12_factor(A)
    assert skipped == 0
    K = oracle.num_reflectors(m, n)
    assert np.all(up[K:] == 0)
    R = r_full(F)
    # backward error ||A - QR|| / ||A||
    QR = oracle.apply_q(F, up, R)
    assert np.linalg.norm(A - QR) / np.linalg.norm(A) <= 10 * m * U
    # orthogonality of the product of the reflectors
    Q = q_explicit(F, up)
    assert np.linalg.norm(Q.T @ Q - np.eye(m)) <= 10 * m * U
    # Q^T A is upper triangular and equals R
    QtA = oracle.apply_qt(F, up, A)
    assert np.max(np.abs(np.tril(QtA, -1))) <= 10 * m * U * np.max(np.abs(A))
    np.testing.assert_allclose(QtA[:n], R[:n], atol=10 * m * U * np.max(np.abs(A)))
    # column norms preserved: sum_i R_ij^2 = sum_i A_ij^2
    np.testing.assert_allclose((R ** 2).sum(0), (A ** 2).sum(0), rtol=10 * m * U)
    # H12 identity v^T v = -2 b for every reflector
    V = oracle.reflector_vectors(F, up)
    for k in range(K):
        b_k = up[k] * F[k, k]
        assert b_k < 0
        assert abs(V[:, k] @ V[:, k] + 2 * b_k) <= 10 * m * U * abs(b_k)


@pytest.mark.parametrize("m,n", [(8, 3), (40, 40), (64, 17)])
def test_qt_then_q_is_identity(m, n):
    A, b = workloads.gaussian(m, n, seed=7 + m + n)
    F, up, _ = oracle.h12_factor(A)
    B = workloads.gaussian_rhs(m, 3, seed=m)
    QtB = oracle.apply_qt(F, up, B)
    np.testing.assert_allclose(np.linalg.norm(QtB, axis=0), np.linalg.norm(B, axis=0),
                               rtol=10 * m * U)
    np.testing.assert_allclose(oracle.apply_q(F, up, QtB), B, atol=10 * m * U * np.abs(B).max())


# ----------------------------------------------------------------------------
# library cross-checks (run as checkers only)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("m,n", [(6, 6), (30, 12), (64, 64), (64, 9), (256, 128)])
def test_lapack_cross_check(m, n):
    A, b = workloads.gaussian(m, n, seed=1 if (m, n) == (256, 128) else m * 31 + n)
    x, F, up, qtb, status = oracle.lstsq(A, b)
    assert status == 0
    R_lapack = np.linalg.qr(A, mode="r")
    kappa = np.linalg.cond(A)
    np.testing.assert_allclose(np.abs(np.diag(F)[:n]), np.abs(np.diag(R_lapack)),
                               rtol=100 * kappa * m * U)
    # R agrees with LAPACK's up to the sign of each row
    s = np.sign(np.diag(F)[:n]) * np.sign(np.diag(R_lapack))
    np.testing.assert_allclose(np.triu(F[:n, :n]), s[:, None] * R_lapack,
                               atol=100 * kappa * m * U * np.abs(A).max())
    x_lapack = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.linalg.norm(x - x_lapack) <= 1e3 * (kappa + kappa ** 2) * 2.0 ** -52 * np.linalg.norm(x_lapack)
    # the residual norm is the LS residual
    np.testing.assert_allclose(oracle.residual_norm(qtb, n), np.linalg.norm(b - A @ x_lapack),
                               rtol=1e-10, atol=1e3 * kappa * m * U * np.linalg.norm(b))


def test_solve_r_matches_triangular_solve():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(5)
    n = 50
    R = np.triu(rng.standard_normal((n, n))) + 4 * np.eye(n)
    C = rng.standard_normal((n, 3))
    X, status = oracle.solve_r(R, C)
    assert status == 0
    np.testing.assert_allclose(X, scipy_linalg.solve_triangular(R, C, lower=False),
                               rtol=1e-12, atol=1e-12)


# ----------------------------------------------------------------------------
# special cases with closed forms
# ----------------------------------------------------------------------------
def test_upper_triangular_tall_gives_minus_a():
    """For x = (a_kk, 0, .., 0): cl = -a_kk if a_kk > 0 else +|a_kk| ... in both
    cases R_kk = -a_kk, up_k = 2 a_kk and every row of R flips sign: R = -A."""
    rng = np.random.default_rng(3)
    n, m = 6, 9
    T = np.triu(rng.standard_normal((n, n)))
    T[np.diag_indices(n)] = rng.choice([-1.0, 1.0], n) * rng.uniform(0.5, 2.0, n)
    A = np.vstack([T, np.zeros((m - n, n))])
    F, up, _ = oracle.h12_factor(A)
    close(np.triu(F[:n]), -T, ulps=16)
    close(up, 2 * np.diag(T), ulps=4)
    assert np.all(np.tril(F, -1) == 0)


@pytest.mark.parametrize("n,m_eq", [(1, 0), (6, 0), (6, 3), (40, 25), (120, 7)])
def test_stacked_top_block_stays_exactly_zero(n, m_eq):
    """For A = [L^T; C] the reflector of column k has zeros in rows k+1..n-1 and
    no reflector changes those rows: after the factorization the strictly
    lower part of the top n x n block is still exactly zero (the fact the
    structure-aware factorization rests on), and R^T R = A^T A."""
    A, _ = workloads.slsqp_stack(n, m_eq, seed=n + 13 * m_eq)
    assert np.all(np.tril(A[:n], -1) == 0.0)
    F, up, skipped = oracle.h12_factor(A)
    assert skipped == 0
    assert np.all(np.tril(F[:n], -1) == 0.0)
    R = np.triu(F[:n])
    G = A.T @ A
    np.testing.assert_allclose(R.T @ R, G, rtol=0, atol=1e-12 * np.abs(G).max())


def test_orthogonal_input_gives_unit_r():
    rng = np.random.default_rng(11)
    Q, _ = np.linalg.qr(rng.standard_normal((20, 20)))
    F, up, _ = oracle.h12_factor(Q[:, :12])
    R = np.triu(F[:12, :12])
    np.testing.assert_allclose(np.abs(R), np.eye(12), atol=1e-14)


def test_zero_column_is_skipped_and_rank_reported():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((7, 4))
    A[:, 2] = 0.0
    # make column 2 zero after the first two reflectors as well: it starts zero
    F, up, skipped = oracle.h12_factor(A)
    assert skipped == 1 and up[2] == 0.0 and F[2, 2] == 0.0
    x, status = oracle.solve_r(F, np.ones(7))
    assert status == oracle.ERANK and x[2] == 0.0


def test_x0_zero_takes_plus_sign():
    """Column (0, 3, 4): x0 = 0 is not > 0, so cl = +5 and up = 0 - 5 = -5."""
    F, up, _ = oracle.h12_factor(np.array([[0.0], [3.0], [4.0]]))
    assert F[0, 0] == 5.0 and up[0] == -5.0
    assert F[1, 0] == 3.0 and F[2, 0] == 4.0


def test_single_column_is_a_norm():
    A = np.array([[3.0], [-4.0], [12.0]])
    F, up, _ = oracle.h12_factor(A)
    assert F[0, 0] == -13.0 and up[0] == 16.0


def test_square_last_column_has_no_reflector():
    A, _ = workloads.gaussian(5, 5, seed=9)
    F, up, _ = oracle.h12_factor(A)
    assert up[4] == 0.0 and oracle.num_reflectors(5, 5) == 4


def test_m_equals_n_plus_one():
    A, b = workloads.gaussian(9, 8, seed=4)
    x, F, up, qtb, status = oracle.lstsq(A, b)
    x_ref = np.linalg.lstsq(A, b, rcond=None)[0]
    np.testing.assert_allclose(x, x_ref, rtol=1e-9)
    assert np.all(up != 0)


@pytest.mark.parametrize("scale", [1e300, 1e-300, 2.0 ** 1000, 2.0 ** -1060])
def test_scaled_norm_does_not_overflow_or_underflow(scale):
    """Reading R5: the column norm is scaled by max|x_i|, so building one
    reflector neither overflows nor underflows where sum x_i^2 would."""
    x = np.array([[3.0], [-4.0], [12.0], [0.0]])
    F, up, _ = oracle.h12_factor(x * scale)
    assert np.isfinite(F[0, 0]) and F[0, 0] != 0
    np.testing.assert_allclose(F[0, 0] / scale, -13.0, rtol=1e-15)
    np.testing.assert_allclose(up[0] / scale, 16.0, rtol=1e-15)


@pytest.mark.parametrize("scale", [1e150, 1e-150])
def test_factor_is_scale_equivariant(scale):
    """R(sA) = s R(A) and up(sA) = s up(A) while the dot products stay in range."""
    A, _ = workloads.gaussian(12, 4, seed=6)
    F1, up1, _ = oracle.h12_factor(A)
    F2, up2, _ = oracle.h12_factor(A * scale)
    np.testing.assert_allclose(np.triu(F2[:4]) / scale, np.triu(F1[:4]), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(up2 / scale, up1, rtol=1e-12)


def test_empty_shapes():
    F, up, sk = oracle.h12_factor(np.zeros((3, 0)))
    assert F.shape == (3, 0) and up.shape == (0,)
    x, st = oracle.solve_r(np.zeros((0, 0)), np.zeros((0,)))
    assert st == 0 and x.shape == (0,)
