"""GPU tests of the tuning knobs (slqr_set_tuning) and the autotuner
(slqr_autotune): the settings only change how the factorization is blocked
and scheduled, so the result stays within the oracle tolerance of
tests/test_gpu_parity.py under every setting."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from test_gpu_parity import dev, host, factor_tol

pytestmark = pytest.mark.gpu


@pytest.fixture()
def ctx():
    from paper_2506_09463_gb300 import abi, api
    c = api.Context(0)
    yield c
    abi.slqr_set_tuning(0, 0)
    c.close()


def factor_matches_oracle(ctx, m, n, seed):
    A, _ = workloads.gaussian(m, n, seed)
    Ad = dev(A)
    up = torch.empty(n, dtype=torch.float64, device="cuda")
    ctx.factor(Ad, up)
    assert ctx.sync() == 0
    tol, _ = factor_tol(A)
    Fo, upo, _ = oracle.h12_factor(A)
    np.testing.assert_allclose(host(Ad), Fo, rtol=0, atol=tol)
    np.testing.assert_allclose(host(up), upo, rtol=0, atol=tol)


@pytest.mark.parametrize("nb,rows", [(32, 64), (64, 96), (64, 256), (32, 0)])
def test_settings_keep_parity(ctx, nb, rows):
    from paper_2506_09463_gb300 import abi
    abi.slqr_set_tuning(nb, rows)
    assert abi.slqr_panel_width(1500, 700) == nb
    factor_matches_oracle(ctx, 1500, 700, seed=nb + rows)


def test_autotune(ctx):
    from paper_2506_09463_gb300 import abi
    st, ms, width, rows = abi.slqr_autotune(ctx.ctx, 1500, 1000)
    assert st == 0, abi.slqr_last_error(ctx.ctx)
    assert ms > 0 and width in (32, 64) and rows in (0, 64, 96, 128, 192, 256)
    assert abi.slqr_panel_width(1500, 1000) == width          # kept for this shape
    assert abi.slqr_panel_width(1500, 999) == 64              # other shapes: defaults
    assert abi.slqr_panel_width(1500, 200) == 32
    factor_matches_oracle(ctx, 1500, 1000, seed=77)
    abi.slqr_set_tuning(0, 0)                                  # forgets the table
    assert abi.slqr_panel_width(1500, 1000) == 64
    assert abi.slqr_autotune(ctx.ctx, 10, 20)[0] == abi.SLQR_EINVAL


def test_autotune_tiny(ctx):
    from paper_2506_09463_gb300 import abi
    st, ms, width, rows = abi.slqr_autotune(ctx.ctx, 40, 17)
    assert st == 0 and width == 32
