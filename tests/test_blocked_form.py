"""The blocked form of Alg. 2 that every trailing-update kernel applies (CPU).

The GPU path applies a panel of reflectors at once in compact-WY form,
    H_{k0+nb-1} ... H_{k0} X = X - V T^T V^T X,
with V the panel's reflector vectors (as stored: up_k on the diagonal, the
tails below), T upper triangular with T^{-1} = striu(V^T V) + diag(1 / tau)
and tau_k = -1 / b_k, b_k = up_k F[k, k] (the compact-WY store keeps Vtop,
striu(V^T V) and tau).  This is a reading of the block algorithm, not a
formula the paper prints, so it is pinned here against the reflectors of the
oracle applied one at a time (H_k x = x + v_k (v_k^T x) / b_k) and against
the oracle's own Q^T application, panel by panel, for panel widths 8, 32 and
64 and a last panel narrower than the rest.  The look-ahead update, the
tiled and tensor-core updates and the Q application all compute this form.
"""
import numpy as np
import pytest

import oracle
import workloads

U = 2.0 ** -53


def panel_wy(V, b, k0, k1):
    """V_p, T^T for reflectors [k0, k1): T^{-1} = striu(V^T V) + diag(1 / tau)."""
    Vp = V[:, k0:k1]
    tau = -1.0 / b[k0:k1]
    Tinv = np.triu(Vp.T @ Vp, 1) + np.diag(1.0 / tau)
    T = np.linalg.solve(Tinv, np.eye(k1 - k0))
    return Vp, T


@pytest.mark.parametrize("m,n,nb", [(50, 20, 8), (97, 64, 32), (200, 130, 64), (300, 300, 64)])
def test_compact_wy_panels_match_the_reflectors_one_at_a_time(m, n, nb):
    A, _ = workloads.gaussian(m, n, seed=3 * m + n)
    F, up, skipped = oracle.h12_factor(A)
    assert skipped == 0
    V = oracle.reflector_vectors(F, up)
    K = V.shape[1]
    b = up[:K] * np.diag(F)[:K]
    X0 = workloads.gaussian_rhs(m, 5, seed=m + nb)
    X = X0.copy()
    tol = 100 * m * U * max(1.0, float(np.abs(X0).max()))
    for k0 in range(0, K, nb):
        k1 = min(K, k0 + nb)
        Vp, T = panel_wy(V, b, k0, k1)
        assert np.allclose(np.tril(T, -1), 0.0)
        blocked = X - Vp @ (T.T @ (Vp.T @ X))
        one_by_one = X.copy()
        for k in range(k0, k1):
            one_by_one += np.outer(V[:, k], V[:, k] @ one_by_one) / b[k]
        assert np.max(np.abs(blocked - one_by_one)) <= tol, (k0, np.max(np.abs(blocked - one_by_one)))
        X = one_by_one
    # all panels together: the oracle's Q^T
    assert np.max(np.abs(X - oracle.apply_qt(F, up, X0))) <= tol


@pytest.mark.parametrize("m,n,nb", [(64, 40, 16), (129, 65, 64)])
def test_compact_wy_q_is_the_transpose_form(m, n, nb):
    """Q X (panels in reverse, X - V T V^T X) undoes Q^T X."""
    A, _ = workloads.gaussian(m, n, seed=m * n)
    F, up, _ = oracle.h12_factor(A)
    V = oracle.reflector_vectors(F, up)
    K = V.shape[1]
    b = up[:K] * np.diag(F)[:K]
    X0 = workloads.gaussian_rhs(m, 3, seed=n)
    Y = oracle.apply_qt(F, up, X0)
    starts = list(range(0, K, nb))
    for k0 in reversed(starts):
        k1 = min(K, k0 + nb)
        Vp, T = panel_wy(V, b, k0, k1)
        Y = Y - Vp @ (T @ (Vp.T @ Y))
    assert np.max(np.abs(Y - X0)) <= 100 * m * U * max(1.0, float(np.abs(X0).max()))
    np.testing.assert_allclose(oracle.apply_q(F, up, oracle.apply_qt(F, up, X0)), X0,
                               atol=100 * m * U * max(1.0, float(np.abs(X0).max())))
