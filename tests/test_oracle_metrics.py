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


# ---- pins of the bound helpers (Theorem 1, Lemma 6 and phi, App. A) and of
# principal_angles, by values worked out by hand from the statements

def test_phi_hand_worked():
    """phi of Theorem 1 at l = 4, j = 2, k = 3, n = 5, beta = e/3, gamma = sqrt(2):
    l - j + 1 = 3 and e / (3 beta) = 1, so the first term is 1 / sqrt(6 pi);
    2 gamma^2 / e^(gamma^2 - 1) = 4/e and 4 gamma (gamma^2 - 1) = 4 sqrt(2), so the
    second is (16 / (e^2 sqrt(2 pi)) + 256 / (2 e^4 sqrt(pi))) / (4 sqrt(2)).
    The decimal values were evaluated at 40 digits."""
    import math

    got = metrics.phi(4, 2, 5, 3, math.e / 3, math.sqrt(2.0))
    assert abs(got - 0.6168591950070394712949970033) < 1e-14


def test_theorem1_rhs_hand_worked_shift_at_sigma_j1():
    """A shift equal to sigma_{j+1}^2 makes the first product of Theorem 1
    vanish: sigma = (4, 3, 2, 1), j = 1, k = 3, l = 4, n = 5, beta = gamma = 2,
    alpha_1 = 9. Then P1 = 0, P2 = ((1 - 9) / (16 - 9))^2 = 64/49 and the
    bound is 2 sqrt(3^2 + (2*4*2*16*64/49 + 1) * 1^2) = 2 sqrt(16874) / 7."""
    sigma = np.array([4.0, 3.0, 2.0, 1.0, 0.5])
    got = metrics.theorem1_rhs(sigma, [9.0], 4, 1, 5, 3, 2.0, 2.0)
    assert abs(got - 37.11427471681350316854814681) < 1e-12


def test_lemma6_rhs_hand_worked():
    """Lemma 6 at sigma = (4, 3, 2, 1), p = 1, j = 1, k = 3, l = 4, n = 5,
    beta = gamma = 2: (2*16*16*(3/4)^4 + 1) * 9 = 163 * 9 = 1467 and
    (2*4*2*16*(1/4)^4 + 1) * 1 = 2, so the bound is 2 sqrt(1469)."""
    sigma = np.array([4.0, 3.0, 2.0, 1.0, 0.5])
    got = metrics.lemma6_rhs(sigma, 1, 4, 1, 5, 3, 2.0, 2.0)
    assert abs(got - 76.65507158694720050218845810) < 1e-12


@pytest.mark.parametrize("p", [1, 2, 5])
def test_theorem1_with_zero_shifts_is_lemma6(p):
    """With every alpha_c = 0 each factor of Theorem 1's products is
    (sigma_{j+1}^2 / sigma_j^2)^2, so p of them give (sigma_{j+1} / sigma_j)^{4p}:
    the shifted bound reduces to the unshifted one of Lemma 6."""
    rng = np.random.default_rng(p)
    sigma = np.sort(rng.uniform(0.1, 10.0, 40))[::-1]
    for j, k, l, n in [(1, 5, 8, 40), (3, 10, 15, 40), (7, 12, 20, 33)]:
        a = metrics.theorem1_rhs(sigma, [0.0] * p, l, j, n, k, 1.5, 1.2)
        b = metrics.lemma6_rhs(sigma, p, l, j, n, k, 1.5, 1.2)
        assert abs(a - b) <= 1e-12 * b


@pytest.mark.parametrize("theta", [0.0, 1e-6, 0.3, np.pi / 2])
def test_principal_angles_closed_form(theta):
    """span(e1, e2) against span(e1, cos(theta) e2 + sin(theta) e3) has
    principal angles 0 and theta; the columns need not be orthonormal
    (they are scaled and mixed here)."""
    n = 6
    e = np.eye(n)
    X = np.stack([3.0 * e[0], e[0] + 2.0 * e[1]], axis=1)
    Y = np.stack([-e[0], np.cos(theta) * e[1] + np.sin(theta) * e[2]], axis=1)
    ang = metrics.principal_angles(X, Y)
    assert ang.shape == (2,)
    assert abs(ang[0]) < 1e-7  # arccos near 1 resolves angles to about 1e-8
    assert abs(ang[1] - theta) < 1e-7 + 1e-12 * theta


def test_principal_angles_orthogonal_complement():
    """Two subspaces that share nothing give angles pi/2 throughout."""
    e = np.eye(5)
    ang = metrics.principal_angles(e[:, :2], e[:, 2:4])
    assert np.allclose(ang, np.pi / 2, atol=1e-15)
