"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (FP64, u = 2^-53):
  * factor (R, reflector tails, up), elementwise:
        |F_gpu - F_oracle| <= 4 sqrt(m) u kappa(A) max_j ||a_j||
    Each result is the exact factorization of a perturbed A + dA with
    ||da_j|| <~ sqrt(m) u ||a_j|| (Householder QR is backward stable; the
    rounding errors of its length-m dot products add up like a random walk,
    in the oracle's sequential order as in the GPU's blocked one), and the
    first-order QR perturbation bound ||dR|| <= sqrt(2) kappa ||dA|| (the
    reflector columns move likewise) makes the two differ by at most about
    2 sqrt(2) kappa sqrt(m) u max ||a_j||.
  * Q^T b, elementwise: <= 4 sqrt(m) u kappa ||b|| by the same argument.
  * LS solution: ||x - x_oracle|| / ||x_oracle|| <= 64 (kappa + kappa^2 ||r|| /
    (||A|| ||x||)) u, the LS forward-error bound for backward errors of a few
    u ||A|| (for a consistent system the kappa u term alone).
  * backward error ||A - QR||_F / ||A||_F <= 1e-12 (the specification's).
The full-size workloads (16384 x 2048, 8192 x 8192) are compared element by
element with oracle outputs computed in background processes
(tests/oracle_outputs.py).  The rounding order differs from the sequential
oracle (blocked sums, power-of-two scaled norms), so nothing here is bitwise.
"""
import numpy as np
import pytest
import torch

import checkers
import oracle
import workloads

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52
U = 2.0 ** -53


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
    m = A.shape[0]
    return 4.0 * np.sqrt(m) * U * kappa * max(1.0, float(np.max(np.linalg.norm(A, axis=0)))), kappa


def x_bound(kappa, A_norm2, r_norm, x_norm):
    """64 (kappa + kappa^2 ||r|| / (||A|| ||x||)) u"""
    return 64.0 * (kappa + kappa ** 2 * r_norm / (A_norm2 * max(x_norm, 1e-300))) * U


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
    np.testing.assert_allclose(qtb, qtbo, rtol=0,
                               atol=4.0 * np.sqrt(m) * U * kappa * np.linalg.norm(b))
    xo, sto = oracle.solve_r(Fo, qtbo)
    r = oracle.residual_norm(qtbo, n)
    bound = x_bound(kappa, np.linalg.norm(A, 2), r, np.linalg.norm(xo))
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
                               atol=4.0 * np.sqrt(m) * U * kappa * np.linalg.norm(B, axis=0).max())
    ctx.solve_r(Ad, Bd)
    assert ctx.sync() == 0
    Xo, _ = oracle.solve_r(Fo, QtBo)
    A2 = np.linalg.norm(A, 2)
    for j in range(B.shape[1]):
        r = np.linalg.norm(QtBo[n:, j])
        err = np.linalg.norm(host(Bd)[:n, j] - Xo[:, j]) / np.linalg.norm(Xo[:, j])
        assert err <= x_bound(kappa, A2, r, np.linalg.norm(Xo[:, j])), (j, err)


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
# full sizes, in the launch configuration the benchmark times, against the
# oracle's outputs element by element (every column)
# --------------------------------------------------------------------------
@pytest.mark.full_oracle("tall", "square")
@pytest.mark.parametrize("name", ["tall", "square"])
def test_full_size(ctx, name):
    import oracle_outputs
    inp = oracle_outputs.inputs(name)
    A, b = inp[0], inp[1]
    B = inp[2] if name == "tall" else np.zeros((A.shape[0], 0))
    m, n = A.shape
    seed = workloads.SEED_TALL if name == "tall" else workloads.SEED_SQUARE
    A0 = dev(A)
    Ad = A0.t().clone().t()
    assert Ad.stride() == (1, m)
    up = torch.empty(n, dtype=torch.float64, device="cuda")
    wy = ctx.wy_buffer(m, n)
    ctx.factor(Ad, up, wy)
    assert ctx.sync() == 0
    # (1) invariants: column norms kept by the orthogonal transform, backward
    #     error ||A - QR|| / ||A|| (independent torch checker)
    R = torch.triu(Ad[:n, :n])
    cn_r, cn_a = (R * R).sum(0), (A0 * A0).sum(0)
    assert float(((cn_r - cn_a).abs() / cn_a).max()) <= 100 * m * EPS
    assert checkers.backward_error_estimate(A0, Ad, up) <= 1e-12
    kappa = checkers.cond_estimate(R)
    A2 = checkers.norm2_estimate(R)
    # (2) Q^T and the back-substitution for b (and 64 right-hand sides), as
    #     the benchmark runs them, with the compact-WY store
    bd = dev(b.reshape(-1, 1))
    ctx.apply_qt(Ad, up, bd, wy=wy)
    qtb = host(bd)[:, 0].copy()
    ctx.solve_r(Ad, bd)
    x = host(bd)[:n, 0].copy()
    Bd = dev(B) if B.shape[1] else None
    if Bd is not None:
        ctx.apply_qt(Ad, up, Bd, wy=wy)
        QtB = host(Bd).copy()
        ctx.solve_r(Ad, Bd)
        X = host(Bd)[:n].copy()
    # (3) consistent system b = A x_true: forward error <= 1e3 kappa 2^-52
    g = torch.Generator(device="cpu").manual_seed(seed)
    x_true = torch.randn(n, 1, generator=g, dtype=torch.float64).cuda()
    bc = (A0 @ x_true).t().contiguous().t()
    ctx.apply_qt(Ad, up, bc, wy=wy)
    ctx.solve_r(Ad, bc)
    assert ctx.sync() == 0
    err = float(torch.linalg.norm(bc[:n] - x_true) / torch.linalg.norm(x_true))
    assert err <= 1e3 * kappa * EPS, (err, kappa)
    F = host(Ad)
    up_h = host(up)
    del Ad, A0, bd, bc, Bd
    torch.cuda.empty_cache()
    # (4) every element of the factorization, Q^T b and x against the oracle
    _, out = oracle_outputs.get(name)
    colmax = float(np.max(np.linalg.norm(A, axis=0)))
    tol_f = 4.0 * np.sqrt(m) * U * kappa * colmax
    for c0 in range(0, n, 1024):                 # column blocks: bounded host memory
        c1 = min(n, c0 + 1024)
        d = float(np.max(np.abs(F[:, c0:c1] - out["F"][:, c0:c1])))
        assert d <= tol_f, (c0, d, tol_f)
    assert float(np.max(np.abs(up_h - out["up"]))) <= tol_f
    qtbs = np.column_stack([qtb, QtB]) if B.shape[1] else qtb[:, None]
    xs = np.column_stack([x, X]) if B.shape[1] else x[:, None]
    bs = np.column_stack([b, B]) if B.shape[1] else b[:, None]
    for j in range(bs.shape[1]):
        tol_q = 4.0 * np.sqrt(m) * U * kappa * np.linalg.norm(bs[:, j])
        assert float(np.max(np.abs(qtbs[:, j] - out["qtb"][:, j]))) <= tol_q, j
        xo = out["x"][:, j]
        r = np.linalg.norm(out["qtb"][n:, j])
        rel = np.linalg.norm(xs[:, j] - xo) / np.linalg.norm(xo)
        assert rel <= x_bound(kappa, A2, r, np.linalg.norm(xo)), (j, rel)
