"""Pins of the oracle's accuracy metrics (Sec. 4) by closed forms: each metric
is zero on the exact truncated SVD and takes a value fixed by the spectrum on
a planted perturbation of it."""
import numpy as np
import pytest

import datagen
from oracle import metrics


def _case(m=120, n=80, seed=5):
    sv = np.linspace(10.0, 1.0, n) ** 2  # distinct, decaying
    A = datagen.dense_with_spectrum(m, n, sv, seed)
    U, S, Vt = np.linalg.svd(A, full_matrices=False)
    return A, U, S, Vt.T


def test_exact_truncated_svd_scores_zero():
    A, U, S, V = _case()
    k = 12
    assert metrics.eps_pve(A, U, S, k) < 1e-12
    assert metrics.eps_sigma(S, S, k) == 0.0
    assert metrics.eps_res(A, U, S, V, S, k) < 1e-12
    assert abs(metrics.eps_spec(A, U, S, V, S, k)) < 1e-12


@pytest.mark.parametrize("d", [1e-3, 0.9])
def test_scaled_singular_values(d):
    """S_hat = (1 + d) sigma on exact vectors: eps_sigma = d, eps_res = d
    (A^T u_i - (1 + d) sigma_i v_i = -d sigma_i v_i), eps_PVE = 0, and the
    residual's norm is max(d sigma_1, sigma_{k+1}) (the second case makes the
    first term the larger)."""
    A, U, S, V = _case()
    k = 10
    Sh = S * (1 + d)
    assert abs(metrics.eps_sigma(Sh, S, k) - d) < 1e-12
    assert abs(metrics.eps_res(A, U, Sh, V, S, k) - d) < 1e-10
    assert metrics.eps_pve(A, U, S, k) < 1e-12
    want = (max(d * S[0], S[k]) - S[k]) / S[k]
    assert (want > 0.1) == (d > 0.5)
    assert abs(metrics.eps_spec(A, U, Sh, V, S, k) - want) < 1e-10


def test_swapped_vector():
    """The k-th triplet replaced by the (k+1)-th: eps_PVE = (sigma_k^2 -
    sigma_{k+1}^2) / sigma_{k+1}^2, and the residual keeps sigma_k, so
    eps_spec = (sigma_k - sigma_{k+1}) / sigma_{k+1}."""
    A, U, S, V = _case()
    k = 9
    Uh, Sh, Vh = U.copy(), S.copy(), V.copy()
    Uh[:, k - 1], Sh[k - 1], Vh[:, k - 1] = U[:, k], S[k], V[:, k]
    assert abs(metrics.eps_pve(A, Uh, S, k) - (S[k - 1] ** 2 - S[k] ** 2) / S[k] ** 2) < 1e-9
    assert abs(metrics.eps_spec(A, Uh, Sh, Vh, S, k) - (S[k - 1] - S[k]) / S[k]) < 1e-10


def test_zero_approximation():
    """U S V^T = 0: the residual is A, so eps_spec = (sigma_1 - sigma_{k+1}) / sigma_{k+1}."""
    A, U, S, V = _case()
    k = 7
    Z = np.zeros_like(S)
    assert abs(metrics.eps_spec(A, U, Z, V, S, k) - (S[0] - S[k]) / S[k]) < 1e-10
    assert abs(metrics.eps_sigma(Z, S, k) - 1.0) < 1e-15
