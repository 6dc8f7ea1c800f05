"""Plain FP64 CPU dashSVD: the oracle for the GPU path.

TEST INFRASTRUCTURE: only the tests, the benchmark's CPU-baseline leg and the
smoke check may import this module. It shares no code with the CUDA library.

It follows the paper step by step, with library primitives (scipy's sparse
product, numpy's matmul and LAPACK's symmetric eigensolver) as single steps and
no blocking, fusion or reordering:

* eigSVD (Alg. 3): G = C^T C, [V, D] = eig(G), S = sqrt(D), U = C V S^-1,
  columns put in descending order of S.
* dashSVD with PVE accuracy control for m >= n (Alg. 5): Q from eigSVD(A^T Omega);
  each pass Q <- eigSVD(A^T (A Q) - alpha Q); stop when the surrogate
  per-vector error test (Eq. 19 with the Prop. 3 surrogate Shat + alpha) holds
  for all i <= k; otherwise raise the shift to (Shat_l + alpha)/2 if Shat_l > alpha;
  finally B = A Q and U, S, V from eigSVD(B).
* m < n is handled by running on A^T and swapping U and V (Sec. 3.1, after Alg. 2).

Readings where the paper is silent or ambiguous (each is also listed in the
design notes of the repository):

R1  alpha' (the shift paired with Shat' in the stop test) is the shift used in
    the pass that produced Shat' (``alpha_prev_mode=0``); ``alpha_prev_mode=1``
    takes step 7 literally (alpha' = the already updated alpha).
R2  Shat' = 0 and alpha' = 0 before the first pass, so for tol < 1 the test
    cannot pass at j = 1; the number of passes is the j at which it passes.
R3  The test's denominator Shat_{k+1} + alpha is floored at
    64 * eps * (Shat_1 + alpha) so an exactly rank-k input can stop.
R4  A break leaves Q as computed in that pass (the shift update is skipped).
R6  An eigenvalue at the rounding level of the Gram entries it is made of,
    d_i <= 16 * eps * sum_j V_ji^2 G_jj (eps: unit roundoff of the eigensolver's
    precision), gives a zero column of U in eigSVD instead of dividing by a
    noise-level S_i. The scale is the diagonal of G seen by the eigenvector, not
    d_1: an exactly dependent column of C leaves an eigenvalue of a few eps
    times the norms of the columns it cancels, while a genuine tail direction of
    a skewed spectrum (d_i / d_1 ~ 1e-6 in the shifted passes of Alg. 5, where
    G has the fourth power of sigma) keeps d_i close to its own diagonal entry.
R8  Each eigenvector column is signed so that its largest-magnitude entry
    (lowest index on ties) is positive; ties in D are ordered by lower index.
R10 ``p_max`` counts power iterations (loop passes); passes over A = 2p + 2.
R16 The control without the surrogate (Sec. 4.3, Table 4; the paper gives no
    listing): Eq. 19 on the singular values of B = A Q taken after each pass's
    basis update, sigma^(j-1) for j = 1 being those of the basis of step 2
    (p = 0); the shift update of the pass is made before the test, and on a stop
    the tested B is the B of step 9. Denominator floored as in R3 (squared).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .mlp_ref import features as mlp_features
from .philox import gaussian_block

EPS64 = np.finfo(np.float64).eps
NULL_FACTOR = 16.0  # reading R6


def _canonical_order_and_sign(d: np.ndarray, V: np.ndarray):
    """Descending order of d (ties: lower original index first) and column signs
    such that each column's largest-|.| entry (lowest index on ties) is positive."""
    l = d.size
    order = np.lexsort((np.arange(l), -d))
    d = d[order]
    V = V[:, order].copy()
    piv = np.argmax(np.abs(V), axis=0)  # first index of the maximum
    sgn = np.where(V[piv, np.arange(l)] < 0, -1.0, 1.0)
    V *= sgn[None, :]
    return d, V


def eigsvd(C: np.ndarray, eps: float = EPS64):
    """eigSVD (Alg. 3) of a tall matrix C (rows >= cols).

    Returns U (rows x l), S (l, descending), V (l x l) with C ~= U diag(S) V^T, and
    the mask of null columns (reading R6).
    """
    C = np.asarray(C, dtype=np.float64)
    l = C.shape[1]
    G = C.T @ C
    d, V = np.linalg.eigh(G)  # symmetric eigensolver, ascending
    d, V = _canonical_order_and_sign(d, V)
    scale = (V * V).T @ np.diag(G)  # sum_j V_ji^2 G_jj per eigenvector i
    null = d <= NULL_FACTOR * eps * scale
    S = np.sqrt(np.maximum(d, 0.0))
    inv = np.where(null, 0.0, 1.0 / np.where(null, 1.0, S))
    U = C @ (V * inv[None, :])
    return U, S, V, null


@dataclass
class PassRecord:
    """What one power-iteration pass saw (Alg. 5, steps 4-7)."""

    j: int
    alpha_used: float  # shift in C = A^T A Q - alpha Q
    S: np.ndarray  # Shat, singular values of C (descending)
    ratio: float  # max_{i<=k} |Shat'_i + alpha' - Shat_i - alpha| / denom
    stopped: bool
    alpha_next: float  # shift after step 6
    Q_in: np.ndarray | None = None  # Q before the pass (kept only if asked)


@dataclass
class Result:
    U: np.ndarray  # m x k
    S: np.ndarray  # k
    V: np.ndarray  # n x k
    passes: int
    converged: bool
    alpha: float
    transposed: bool
    trace: list = field(default_factory=list)
    Q: np.ndarray | None = None  # final Q (n x l, on the working side)


def pve_ratio(S_prev, alpha_prev, S, alpha, k):
    """max_{i<=k} |S'_i + alpha' - S_i - alpha| / max(S_{k+1} + alpha, floor)  (Alg. 5 step 5, R3)."""
    denom = max(S[k] + alpha, 64.0 * EPS64 * (S[0] + alpha))
    if denom <= 0.0:
        return np.inf
    return float(np.max(np.abs(S_prev[:k] + alpha_prev - S[:k] - alpha)) / denom)


def next_shift(S_l, alpha, f=1.0):
    """Alg. 5 step 6: alpha <- (Shat_l + alpha) / 2 if Shat_l > alpha (the safe
    bound of Prop. 1); the learned form takes the fraction f of it, clamped to
    [0, bound], and the bound itself for a non-finite f."""
    bound = 0.5 * (S_l + alpha) if S_l > alpha else alpha
    return min(max(f * bound, 0.0), bound) if np.isfinite(f) else bound


def direct_pve_ratio(Sd_prev, Sd, k):
    """max_{i<=k} |s'_i^2 - s_i^2| / max(s_{k+1}^2, floor): Eq. 19 of
    Sec. 3.2 on singular values s of B = A Q (this pass) and s' (the pass
    before), with the floor of R3 at the squared scale (reading R16)."""
    denom = max(Sd[k] ** 2, 64.0 * EPS64 * Sd[0] ** 2)
    if denom <= 0.0:
        return np.inf
    return float(np.max(np.abs(Sd_prev[:k] ** 2 - Sd[:k] ** 2)) / denom)


def dashsvd(
    A,
    k: int,
    s: int,
    p_max: int,
    tol: float,
    seed: int,
    alpha_prev_mode: int = 0,
    shift=True,
    keep_q: bool = False,
    Omega: np.ndarray | None = None,
    policy=None,
    pve_mode: str = "surrogate",
) -> Result:
    """dashSVD with PVE accuracy control (Alg. 5) in FP64.

    ``A`` is a scipy sparse matrix (or dense array). ``tol <= 0`` disables the
    stop test, which gives the fixed-p dashSVD of Alg. 4. ``shift=False`` keeps
    alpha = 0, which is the basic randomized SVD with eigSVD orthonormalization
    (Alg. 1 in the m >= n form); ``shift="fixed"`` takes the first pass's shift
    (Shat_l / 2) and keeps it (the fixed-shift variant Alg. 2* of Sec. 4). ``Omega`` overrides the Philox block.
    ``policy`` (learned form) maps the features of a pass (``mlp_ref.features``)
    to (f, o_1): the next shift is f times the plain rule's value, clamped to
    [0, that value], and o_1 > 0 stops the run from pass 2 on while the
    surrogate ratio is at most 3 tol.
    ``pve_mode="direct"`` runs the accuracy control without the surrogate
    (the comparison of Sec. 4.3, Table 4): after each pass the singular values
    of B = A Q are computed and Eq. 19 is applied to them
    literally, sigma^(j) against sigma^(j-1), sigma^(0) being those of the
    basis before the first pass (p = 0); the shift rule is unchanged.
    """
    import scipy.sparse as sp

    A = sp.csr_matrix(A, dtype=np.float64) if not sp.issparse(A) else A.astype(np.float64).tocsr()
    m, n = A.shape
    transposed = m < n
    if transposed:
        A = A.T.tocsr()
        m, n = n, m
    l = k + s
    if k < 1 or s < 1 or l > n:
        raise ValueError("need k >= 1, s >= 1 and k + s <= min(m, n)")
    At = A.T.tocsr()

    if pve_mode not in ("surrogate", "direct"):
        raise ValueError("pve_mode is 'surrogate' or 'direct'")
    direct = pve_mode == "direct"
    if direct and policy is not None:
        raise ValueError("the learned policy works on the surrogate")
    Om = gaussian_block(seed, m, l) if Omega is None else np.asarray(Omega, dtype=np.float64)
    Q, _, _, _ = eigsvd(At @ Om)  # step 2
    Sd_prev = eigsvd(A @ Q)[1] if direct else None  # sigma^(0): singular values of A Q_0
    alpha = 0.0
    alpha_prev = 0.0
    ratio_prev = 0.0
    S_prev = np.zeros(l)
    trace = []
    passes = 0
    converged = False
    for j in range(1, p_max + 1):  # step 3
        Q_in = Q.copy() if keep_q else None
        C = At @ (A @ Q) - alpha * Q  # step 4
        Q, S, _, _ = eigsvd(C)
        passes = j
        ratio = pve_ratio(S_prev, alpha_prev, S, alpha, k)
        stop = tol > 0 and ratio <= tol and not direct  # step 5
        f = 1.0
        if policy is not None:
            x = mlp_features(S, alpha, ratio, ratio_prev if j > 1 else ratio, j, p_max, tol, k)
            f, o1 = policy(x)
            stop = stop or (tol > 0 and j >= 2 and ratio <= 3.0 * tol and o1 > 0.0)
        if stop:
            trace.append(PassRecord(j, alpha, S, ratio, True, alpha, Q_in))
            converged = True
            break
        alpha_used = alpha
        ratio_prev = ratio
        if shift == "fixed":  # Alg. 2*: alpha = sigma_l(A A^T Q) / 2 from the first pass, then fixed
            if j == 1:
                alpha = 0.5 * S[l - 1]
        elif shift:  # step 6 (learned form: a fraction of the same bound)
            alpha = next_shift(S[l - 1], alpha, f)
        S_prev = S  # step 7
        alpha_prev = alpha_used if alpha_prev_mode == 0 else alpha
        if direct:  # sigma^(j) of B = A Q against sigma^(j-1)
            Sd = eigsvd(A @ Q)[1]
            ratio = direct_pve_ratio(Sd_prev, Sd, k)
            Sd_prev = Sd
            if tol > 0 and ratio <= tol:
                trace.append(PassRecord(j, alpha_used, S, ratio, True, alpha, Q_in))
                converged = True
                break
        trace.append(PassRecord(j, alpha_used, S, ratio, False, alpha, Q_in))

    B = A @ Q  # step 9
    Ub, Sb, Vb, _ = eigsvd(B)  # step 10
    U = Ub[:, :k]  # step 11
    S = Sb[:k]
    V = Q @ Vb[:, :k]
    if transposed:
        U, V = V, U
    return Result(U, S, V, passes, converged, alpha, transposed, trace, Q)
