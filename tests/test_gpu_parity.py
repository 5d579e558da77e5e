"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (FP64, u = 2^-53, eps = 2^-52):
  * factor (R, reflector tails, up), elementwise:
        |F_gpu - F_oracle| <= 1e3 * kappa(A) * eps * max_j ||a_j||
    Both results are backward stable; the QR perturbation bound
    ||dR|| <~ sqrt(2) kappa ||dA|| turns backward errors of ~sqrt(m) u ||A||
    into forward differences well inside this.
  * Q^T b: |d| <= 1e3 * kappa * eps * ||b||.
  * LS solution: ||x - x_oracle|| / ||x_oracle|| <= 1e3 * (kappa + kappa^2 *
    ||r|| / (||A|| ||x||)) * eps (the LS forward-error bound; for a consistent
    system it is the 1e3 kappa 2^-52 bound of the specification).
  * backward error ||A - QR||_F / ||A||_F <= 1e-12.
The rounding order differs from the sequential oracle (blocked sums, power-
of-two scaled norms), so nothing here is bitwise.
"""
import numpy as np
import pytest
import torch

import checkers
import oracle
import workloads

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52


@pytest.fixture(scope="module")
def ctx():
    from paper_2506_09463_gb300 import api
    c = api.Context(0)
    yield c
    c.close()


def dev(a):
    """Column-major float64 CUDA copy of a numpy array (strides (1, m))."""
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        return torch.from_numpy(a.copy()).cuda()
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()


def host(t):
    return t.detach().cpu().numpy()


def factor_tol(A):
    kappa = np.linalg.cond(A) if min(A.shape) > 0 else 1.0
    return 1e3 * kappa * EPS * max(1.0, float(np.max(np.linalg.norm(A, axis=0)))), kappa


def run_gpu(ctx, A, b, nrhs_extra=0, use_wy=True, lda_pad=0):
    m, n = A.shape
    if lda_pad:
        big = np.zeros((m + lda_pad, n))
        big[:m] = A
        Ad = dev(big)[:m]
    else:
        Ad = dev(A)
    up = torch.empty(n, dtype=torch.float64, device="cuda")
    wy = ctx.wy_buffer(m, n) if use_wy else None
    ctx.factor(Ad, up, wy)
    bd = dev(b.reshape(-1, 1))
    ctx.apply_qt(Ad, up, bd, wy=wy)
    qtb = host(bd)[:, 0].copy()
    ctx.solve_r(Ad, bd)
    st = ctx.sync()
    return host(Ad), host(up), qtb, host(bd)[:n, 0], st


def check_against_oracle(A, b, F, up, qtb, x):
    m, n = A.shape
    tol, kappa = factor_tol(A)
    Fo, upo, _ = oracle.h12_factor(A)
    np.testing.assert_allclose(F, Fo, rtol=0, atol=tol)
    np.testing.assert_allclose(up, upo, rtol=0, atol=tol)
    qtbo = oracle.apply_qt(Fo, upo, b)
    np.testing.assert_allclose(qtb, qtbo, rtol=0, atol=1e3 * kappa * EPS * np.linalg.norm(b))
    xo, sto = oracle.solve_r(Fo, qtbo)
    r = oracle.residual_norm(qtbo, n)
    bound = 1e3 * (kappa + kappa ** 2 * r / (np.linalg.norm(A, 2) * max(np.linalg.norm(xo), 1e-300))) * EPS
    assert np.linalg.norm(x - xo) <= bound * np.linalg.norm(xo) + 1e-300


# --------------------------------------------------------------------------
# small and ragged shapes, against the oracle element by element
# --------------------------------------------------------------------------
SHAPES = [
    (256, 128),      # the 256 x 128 single-problem workload (seed 1)
    (1, 1), (2, 1), (3, 2), (2, 2), (33, 17), (65, 65), (97, 96),
    (300, 200), (257, 256),          # panel width 32, several panels, ragged
    (600, 300), (1000, 513),         # panel width 64, ragged last panel
    (4096, 40), (5000, 300),         # tall: many CTAs in the panel kernel
    (1500, 1000),
]


@pytest.mark.parametrize("m,n", SHAPES)
def test_parity_with_oracle(ctx, m, n):
    seed = workloads.SEED_SMALL if (m, n) == (256, 128) else 1000 + m + 7 * n
    A, b = workloads.gaussian(m, n, seed)
    F, up, qtb, x, st = run_gpu(ctx, A, b)
    assert st == 0
    check_against_oracle(A, b, F, up, qtb, x)


@pytest.mark.parametrize("use_wy", [True, False])
def test_apply_qt_many_rhs(ctx, use_wy):
    m, n = 700, 450
    A, _ = workloads.gaussian(m, n, 11)
    B = workloads.gaussian_rhs(m, 64, 11)
    Ad = dev(A)
    up = torch.empty(n, dtype=torch.float64, device="cuda")
    wy = ctx.wy_buffer(m, n)
    ctx.factor(Ad, up, wy)
    Bd = dev(B)
    ctx.apply_qt(Ad, up, Bd, wy=wy if use_wy else None)
    Fo, upo, _ = oracle.h12_factor(A)
    QtBo = oracle.apply_qt(Fo, upo, B)
    tol, kappa = factor_tol(A)
    np.testing.assert_allclose(host(Bd), QtBo, rtol=0,
                               atol=1e3 * kappa * EPS * np.abs(B).max() * np.sqrt(m))
    ctx.solve_r(Ad, Bd)
    assert ctx.sync() == 0
    Xo, _ = oracle.solve_r(Fo, QtBo)
    err = np.linalg.norm(host(Bd)[:n] - Xo) / np.linalg.norm(Xo)
    assert err <= 1e3 * (kappa + kappa ** 2) * EPS


def test_leading_dimension_padding(ctx):
    A, b = workloads.gaussian(300, 120, 5)
    F, up, qtb, x, st = run_gpu(ctx, A, b, lda_pad=13)
    check_against_oracle(A, b, F, up, qtb, x)


def test_without_wy_store(ctx):
    A, b = workloads.gaussian(513, 300, 6)
    F, up, qtb, x, st = run_gpu(ctx, A, b, use_wy=False)
    check_against_oracle(A, b, F, up, qtb, x)


# --------------------------------------------------------------------------
# hand-worked examples and special cases
# --------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["h12_3x2.txt", "h12_4x3.txt"])
def test_golden_examples_on_gpu(ctx, name):
    from test_oracle_pins import load_golden
    g = load_golden(name)
    A = np.array([[float(v) for v in r] for r in g["A"]])
    b = np.array([float(v) for v in g["b"]])
    F, up, qtb, x, st = run_gpu(ctx, A, b)
    assert st == 0
    at = 16 * EPS * 20
    np.testing.assert_allclose(F, [[float(v) for v in r] for r in g["F"]], rtol=0, atol=at)
    np.testing.assert_allclose(up, [float(v) for v in g["up"]], rtol=0, atol=at)
    np.testing.assert_allclose(qtb, [float(v) for v in g["qtb"]], rtol=0, atol=at)
    np.testing.assert_allclose(x, [float(v) for v in g["x"]], rtol=0, atol=at)


def test_zero_column_skip_and_rank(ctx):
    A, b = workloads.gaussian(80, 40, 8)
    A[:, 9] = 0.0
    F, up, qtb, x, st = run_gpu(ctx, A, b)
    Fo, upo, skipped = oracle.h12_factor(A)
    assert skipped == 1 and up[9] == 0.0 and F[9, 9] == 0.0
    assert st == oracle.ERANK
    assert x[9] == 0.0


def test_x0_zero_sign_rule(ctx):
    A = np.array([[0.0], [3.0], [4.0]])
    F, up, qtb, x, st = run_gpu(ctx, A, np.array([1.0, 2.0, 3.0]))
    assert F[0, 0] == 5.0 and up[0] == -5.0 and F[1, 0] == 3.0 and F[2, 0] == 4.0


def test_upper_triangular_input(ctx):
    rng = np.random.default_rng(3)
    n, m = 70, 90
    T = np.triu(rng.standard_normal((n, n)))
    T[np.diag_indices(n)] = rng.choice([-1.0, 1.0], n) * rng.uniform(0.5, 2.0, n)
    A = np.vstack([T, np.zeros((m - n, n))])
    F, up, qtb, x, st = run_gpu(ctx, A, np.ones(m))
    np.testing.assert_allclose(np.triu(F[:n]), -T, atol=1e-13)
    np.testing.assert_allclose(up, 2 * np.diag(T), atol=1e-13)


def test_square_and_single_column(ctx):
    for (m, n) in [(64, 64), (129, 129), (50, 1)]:
        A, b = workloads.gaussian(m, n, 40 + m)
        F, up, qtb, x, st = run_gpu(ctx, A, b)
        check_against_oracle(A, b, F, up, qtb, x)
        if m == n:
            assert up[-1] == 0.0


def test_empty_and_invalid_arguments(ctx):
    from paper_2506_09463_gb300 import abi
    A = torch.zeros(4, 0, dtype=torch.float64, device="cuda")
    ctx.factor(A)                                   # n = 0: no-op
    Ad = torch.zeros(3, 5, dtype=torch.float64, device="cuda")
    with pytest.raises(abi.SlqrError) as e:
        ctx.factor(Ad.t().contiguous().t())         # m < n
    assert e.value.status == abi.SLQR_EINVAL
    st = abi.slqr_factor(ctx.ctx, 10, 4, Ad.data_ptr(), 5, Ad.data_ptr(), None, 0)
    assert st == abi.SLQR_EINVAL                    # lda < m
    st = abi.slqr_apply_qt(ctx.ctx, 10, 4, Ad.data_ptr(), 10, Ad.data_ptr(), None, -1,
                           Ad.data_ptr(), 10, 0)
    assert st == abi.SLQR_EINVAL                    # nrhs < 0
    st = abi.slqr_factor(ctx.ctx, abi.slqr_max_rows() + 1, 4, Ad.data_ptr(),
                         abi.slqr_max_rows() + 1, Ad.data_ptr(), None, 0)
    assert st == abi.SLQR_EINVAL
    assert ctx.sync() == 0


# --------------------------------------------------------------------------
# full sizes, in the launch configuration the benchmark times
# --------------------------------------------------------------------------
@pytest.mark.parametrize("m,n,seed", [(16384, 2048, workloads.SEED_TALL),
                                      (8192, 8192, workloads.SEED_SQUARE)])
def test_full_size(ctx, m, n, seed):
    A, b = workloads.gaussian(m, n, seed)
    A0 = dev(A)
    Ad = A0.t().clone().t()
    assert Ad.stride() == (1, m)
    up = torch.empty(n, dtype=torch.float64, device="cuda")
    wy = ctx.wy_buffer(m, n)
    ctx.factor(Ad, up, wy)
    assert ctx.sync() == 0
    # (1) sampled outputs: the first 128 columns depend only on A[:, :128]
    p = 128
    Fo, upo, _ = oracle.h12_factor(A[:, :p])
    tol, _ = factor_tol(A[:, :p])
    np.testing.assert_allclose(host(Ad[:, :p]), Fo, rtol=0, atol=tol)
    np.testing.assert_allclose(host(up[:p]), upo, rtol=0, atol=tol)
    # (2) column norms are preserved by the orthogonal transform
    R = torch.triu(Ad[:n, :n])
    cn_r, cn_a = (R * R).sum(0), (A0 * A0).sum(0)
    assert float(((cn_r - cn_a).abs() / cn_a).max()) <= 100 * m * EPS
    # (3) backward error ||A - QR|| / ||A|| (independent torch checker)
    assert checkers.backward_error_estimate(A0, Ad, up) <= 1e-12
    # (4) Q^T with 1 and 64 right-hand sides against the checker
    B = torch.from_numpy(workloads.gaussian_rhs(m, 64, seed)).cuda()
    B = B.t().contiguous().t()
    ref = checkers.apply_qt(Ad, up, B)
    Bd = B.clone().t().contiguous().t()
    ctx.apply_qt(Ad, up, Bd, wy=wy)
    assert float((Bd - ref).abs().max()) <= 1e3 * EPS * float(B.abs().max()) * np.sqrt(m)
    b1 = B[:, :1].clone()
    ctx.apply_qt(Ad, up, b1, wy=wy)
    assert float((b1 - ref[:, :1]).abs().max()) <= 1e3 * EPS * float(B.abs().max()) * np.sqrt(m)
    # (5) consistent system b = A x_true: forward error <= 1e3 kappa 2^-52
    kappa = checkers.cond_estimate(R)
    g = torch.Generator(device="cpu").manual_seed(seed)
    x_true = torch.randn(n, 1, generator=g, dtype=torch.float64).cuda()
    bc = (A0 @ x_true).t().contiguous().t()
    ctx.apply_qt(Ad, up, bc, wy=wy)
    ctx.solve_r(Ad, bc)
    assert ctx.sync() == 0
    err = float(torch.linalg.norm(bc[:n] - x_true) / torch.linalg.norm(x_true))
    assert err <= 1e3 * kappa * EPS, (err, kappa)
    # (6) 64 right-hand sides through the back-substitution vs a torch triangular solve
    X = Bd.clone()
    ctx.solve_r(Ad, X)
    assert ctx.sync() == 0
    Xref = torch.linalg.solve_triangular(R, ref[:n], upper=True)
    rel = float(torch.linalg.norm(X[:n] - Xref) / torch.linalg.norm(Xref))
    assert rel <= 1e3 * kappa * EPS
