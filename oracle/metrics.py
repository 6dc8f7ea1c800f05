"""Accuracy metrics and the paper's error bounds, in FP64.

TEST INFRASTRUCTURE: used by the tests and the benchmark's accuracy check only.

* eps_pve   -- per-vector error (Sec. 4): max_{i<=k} |u_i^T A A^T u_i - uh_i^T A A^T uh_i|
               / sigma_{k+1}(A)^2; for exact singular vectors u_i^T A A^T u_i = sigma_i^2,
               so only ||A^T uh_i||^2 is needed.
* eps_sigma -- max_{i<=k} |sigma_i - sigmah_i| / sigma_i (Sec. 4).
* eps_res   -- max_{i<=k} ||A^T uh_i - sigmah_i vh_i|| / sigma_i (Sec. 4, from Eq. 8).
* eps_spec  -- (||A - Uh Sh Vh^T||_2 - ||A - A_k||_2) / ||A - A_k||_2 with
               ||A - A_k||_2 = sigma_{k+1} (Sec. 4, from Eq. 17); the spectral norm
               of the dense residual by LAPACK's SVD (small matrices).
* theorem1_rhs / lemma6_rhs -- right-hand sides of Theorem 1 (shifted power
  iteration) and Lemma 6 (unshifted), and phi, the failure probability bound
  shared by both (Theorem 1 / Lemma 7).
"""
from __future__ import annotations

import math

import numpy as np


def eps_pve(A, U_hat, sigma_true, k):
    AtU = A.T @ U_hat[:, :k]
    cap = np.einsum("ij,ij->j", AtU, AtU)
    return float(np.max(np.abs(sigma_true[:k] ** 2 - cap)) / sigma_true[k] ** 2)


def eps_sigma(S_hat, sigma_true, k):
    return float(np.max(np.abs(sigma_true[:k] - S_hat[:k]) / sigma_true[:k]))


def eps_res(A, U_hat, S_hat, V_hat, sigma_true, k):
    R = A.T @ U_hat[:, :k] - V_hat[:, :k] * S_hat[None, :k]
    return float(np.max(np.linalg.norm(R, axis=0) / sigma_true[:k]))


def eps_spec(A, U_hat, S_hat, V_hat, sigma_true, k):
    A = A.toarray() if hasattr(A, "toarray") else np.asarray(A, dtype=np.float64)
    R = A - (U_hat[:, :k] * S_hat[None, :k]) @ V_hat[:, :k].T
    return float((np.linalg.norm(R, 2) - sigma_true[k]) / sigma_true[k])


def principal_angles(X, Y):
    """Principal angles (radians, ascending) between span(X) and span(Y)."""
    qx, _ = np.linalg.qr(X)
    qy, _ = np.linalg.qr(Y)
    c = np.linalg.svd(qx.T @ qy, compute_uv=False)
    return np.sort(np.arccos(np.clip(c, -1.0, 1.0)))


def phi(l, j, n, k, beta, gamma):
    """Failure probability bound of Theorem 1 (and Lemma 6)."""
    a = l - j + 1
    t1 = (1.0 / math.sqrt(2 * math.pi * a)) * (math.e / (a * beta)) ** a
    g = 2 * gamma**2 / math.exp(gamma**2 - 1)
    t2 = (1.0 / (4 * gamma * (gamma**2 - 1))) * (
        (1.0 / math.sqrt(math.pi * (n - k))) * g ** (n - k) + (1.0 / math.sqrt(math.pi * l)) * g**l
    )
    return t1 + t2


def theorem1_rhs(sigma, alphas, l, j, n, k, beta, gamma):
    """2 sqrt((2 l^2 b^2 g^2 P1 + 1) s_{j+1}^2 + (2 l (n-k) b^2 g^2 P2 + 1) s_{k+1}^2),
    P1 = prod_c ((s_{j+1}^2 - a_c)/(s_j^2 - a_c))^2, P2 likewise with s_{k+1}
    (sigma is 0-based: sigma[j-1] is sigma_j)."""
    sj, sj1, sk1 = sigma[j - 1], sigma[j], sigma[k]
    p1 = 1.0
    p2 = 1.0
    for a in alphas:
        p1 *= ((sj1**2 - a) / (sj**2 - a)) ** 2
        p2 *= ((sk1**2 - a) / (sj**2 - a)) ** 2
    bg = beta**2 * gamma**2
    return 2.0 * math.sqrt(
        (2 * l * l * bg * p1 + 1) * sj1**2 + (2 * l * (n - k) * bg * p2 + 1) * sk1**2
    )


def lemma6_rhs(sigma, p, l, j, n, k, beta, gamma):
    """Unshifted bound: the products of Theorem 1 become (s_{j+1}/s_j)^{4p} and (s_{k+1}/s_j)^{4p}."""
    sj, sj1, sk1 = sigma[j - 1], sigma[j], sigma[k]
    bg = beta**2 * gamma**2
    return 2.0 * math.sqrt(
        (2 * l * l * bg * (sj1 / sj) ** (4 * p) + 1) * sj1**2
        + (2 * l * (n - k) * bg * (sk1 / sj) ** (4 * p) + 1) * sk1**2
    )
