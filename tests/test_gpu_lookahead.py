"""The fused look-ahead update of the FP32 factorization
(slqr_set_fused_lookahead) against the three-launch update and the oracle.

After each panel of width 64, the next panel's columns are updated by the
panel's reflectors in compact-WY form (Alg. 2 by blocks) before the next panel
is factored.  The fused kernel and the tiled launches compute the same
product with partial sums in different orders, so each mixed-precision solve
is held to the refined-solution tolerance of the mixed-precision tests
against the oracle's FP64 solution, and both settings must need about the
same number of refinement sweeps (a wrong update of the next panel would
leave a factorization that is not backward stable, and the sweeps would stall
or diverge).  Shapes cover 32 and 64 rows per CTA, rows that are not a
multiple of 4 (the scalar tail of the staged slices), a last panel narrower
than 64 (the look-ahead updates fewer than 64 columns), and a matrix too tall
for the fused kernel (more than 256 rows per CTA: the tiled launches run).
"""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def ctx():
    from paper_2506_09463_gb300 import abi, api
    c = api.Context(0)
    yield c
    abi.slqr_set_fused_lookahead(1)
    c.close()


def solve(ctx, A, b, prec, fused):
    from paper_2506_09463_gb300 import abi
    assert abi.slqr_set_fused_lookahead(fused) == abi.SLQR_OK
    m, n = A.shape
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, info = abi.slqr_lstsq_mixed_ex(ctx.ctx, m, n, A.data_ptr(), A.stride(1), b.data_ptr(),
                                       x.data_ptr(), prec,
                                       torch.cuda.current_stream().cuda_stream,
                                       refine=abi.SLQR_REFINE_BJORCK, fp64_fallback=0)
    torch.cuda.synchronize()
    return st, info, x.cpu().numpy()


def check_against_oracle(A, b, x, kappa, label):
    Ah, bh = A.cpu().numpy(), b.cpu().numpy()
    xo = oracle.lstsq(Ah, bh)[0]
    r = np.linalg.norm(bh - Ah @ xo)
    tol = max(1e-10, 64.0 * (kappa + kappa ** 2 * r / (np.linalg.norm(Ah, 2) *
                                                      np.linalg.norm(xo))) * U)
    err = np.max(np.abs(x - xo)) / np.max(np.abs(xo))
    assert err <= tol, (label, err, tol)


@pytest.mark.parametrize("m,n,kappa", [(2048, 512, 1e4), (3001, 700, 1e3), (9000, 320, 1e3),
                                       (39500, 128, 1e2)])
def test_fused_lookahead_mixed_fp32(ctx, m, n, kappa):
    from paper_2506_09463_gb300 import abi
    A, b_cons, x_true, b_rand = workloads.conditioned_device(m, n, kappa, seed=m + n)
    sweeps = {}
    for fused in (1, 0):
        for name, b in (("consistent", b_cons), ("random", b_rand)):
            st, info, x = solve(ctx, A, b, abi.SLQR_FP32, fused)
            assert st == abi.SLQR_OK, (fused, name, st, info)
            assert info["method"] == abi.SLQR_REFINE_BJORCK
            check_against_oracle(A, b, x, kappa, (fused, name))
            sweeps[(fused, name)] = info["sweeps"]
    for name in ("consistent", "random"):
        assert sweeps[(1, name)] <= sweeps[(0, name)] + 1, sweeps
    assert abi.slqr_get_fused_lookahead() == 0
    assert abi.slqr_set_fused_lookahead(1) == abi.SLQR_OK


@pytest.mark.parametrize("prec_name", ["SLQR_TF32", "SLQR_BF16X3"])
def test_fused_lookahead_tensor_core_modes(ctx, prec_name):
    """The look-ahead runs on the FP32 FMA pipe in every mode; the rest of the
    trailing update stays on the tensor cores."""
    from paper_2506_09463_gb300 import abi
    m, n, kappa = 4100, 640, 1e2
    A, b_cons, x_true, b_rand = workloads.conditioned_device(m, n, kappa, seed=31)
    prec = getattr(abi, prec_name)
    for fused in (1, 0):
        st, info, x = solve(ctx, A, b_rand, prec, fused)
        assert st == abi.SLQR_OK, (prec_name, fused, st, info)
        check_against_oracle(A, b_rand, x, kappa, (prec_name, fused))
    abi.slqr_set_fused_lookahead(1)


def test_fused_lookahead_setting_range(ctx):
    from paper_2506_09463_gb300 import abi
    for bad in (-1, 2, 7):
        assert abi.slqr_set_fused_lookahead(bad) == abi.SLQR_EINVAL
    for good in (0, 1):
        assert abi.slqr_set_fused_lookahead(good) == abi.SLQR_OK
        assert abi.slqr_get_fused_lookahead() == good
