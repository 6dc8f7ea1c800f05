"""Pins for the oracle's eigSVD (Alg. 3) and dashSVD (Alg. 4 / Alg. 5).

Nothing here compares the oracle with itself: each test checks it against a
closed form, a different LAPACK routine (gesdd via numpy.linalg.svd, QR), brute
force, or an inequality the paper proves (Prop. 1-3, Theorem 1, its Corollary).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import datagen
import oracle
from oracle import metrics
from oracle.dashsvd_ref import dashsvd, eigsvd


def _sparse(m, n, density, seed):
    rng = np.random.default_rng(seed)
    A = sp.random(m, n, density=density, random_state=rng, data_rvs=rng.standard_normal, format="csr")
    return A


def _abs_col_cos(X, Y):
    Xn = X / np.linalg.norm(X, axis=0)
    Yn = Y / np.linalg.norm(Y, axis=0)
    return np.abs(np.einsum("ij,ij->j", Xn, Yn))


# ----------------------------------------------------------------- eigSVD


def test_eigsvd_orthogonal_columns_closed_form():
    C = np.zeros((5, 3))
    C[0, 1] = 3.0
    C[2, 0] = -2.0
    C[4, 2] = 0.5
    U, S, V, null = eigsvd(C)
    np.testing.assert_allclose(S, [3.0, 2.0, 0.5], rtol=1e-15)
    assert not null.any()
    np.testing.assert_allclose(U @ np.diag(S) @ V.T, C, atol=1e-14)
    # sign rule: largest |entry| of every V column is positive
    assert np.all(V[np.argmax(np.abs(V), axis=0), range(3)] > 0)


def test_eigsvd_matches_gesdd():
    rng = np.random.default_rng(1)
    C = rng.standard_normal((300, 40)) @ np.diag(np.logspace(0, -3, 40))
    U, S, V, null = eigsvd(C)
    Ur, Sr, Vtr = np.linalg.svd(C, full_matrices=False)
    np.testing.assert_allclose(S, Sr, rtol=1e-9)
    assert np.all(np.diff(S) <= 0)
    assert np.min(_abs_col_cos(U, Ur)) > 1 - 1e-6
    assert np.min(_abs_col_cos(V, Vtr.T)) > 1 - 1e-9
    np.testing.assert_allclose(U.T @ U, np.eye(40), atol=1e-6)
    np.testing.assert_allclose((U * S) @ V.T, C, atol=1e-12)


def test_eigsvd_rank_deficient_null_columns():
    rng = np.random.default_rng(2)
    C = rng.standard_normal((100, 5)) @ rng.standard_normal((5, 12))
    U, S, V, null = eigsvd(C)
    assert null.sum() == 7 and not null[:5].any()
    assert np.all(U[:, null] == 0)
    np.testing.assert_allclose(U[:, ~null].T @ U[:, ~null], np.eye(5), atol=1e-10)
    np.testing.assert_allclose(S[:5], np.linalg.svd(C, compute_uv=False)[:5], rtol=1e-11)


# ----------------------------------------------------------------- dashSVD


def test_full_width_subspace_gives_exact_svd():
    """l = n: Q spans R^n after the first eigSVD, so the result is the exact SVD."""
    A = _sparse(90, 14, 0.3, 3)
    k, s = 9, 5
    r = dashsvd(A, k, s, p_max=2, tol=0.0, seed=11)
    Ur, Sr, Vtr = np.linalg.svd(A.toarray(), full_matrices=False)
    np.testing.assert_allclose(r.S, Sr[:k], rtol=1e-12)
    assert np.min(_abs_col_cos(r.U, Ur[:, :k])) > 1 - 1e-10
    assert np.min(_abs_col_cos(r.V, Vtr[:k].T)) > 1 - 1e-10


def test_wide_input_runs_on_transpose():
    A = _sparse(14, 90, 0.3, 4)
    k, s = 9, 5
    r = dashsvd(A, k, s, p_max=1, tol=0.0, seed=12)
    assert r.transposed and r.U.shape == (14, k) and r.V.shape == (90, k)
    Ur, Sr, Vtr = np.linalg.svd(A.toarray(), full_matrices=False)
    np.testing.assert_allclose(r.S, Sr[:k], rtol=1e-12)
    assert np.min(_abs_col_cos(r.U, Ur[:, :k])) > 1 - 1e-10
    assert np.min(_abs_col_cos(r.V, Vtr[:k].T)) > 1 - 1e-10


def test_exact_low_rank_recovery_without_power_iteration():
    rng = np.random.default_rng(5)
    r_true = 5
    A = rng.standard_normal((400, r_true)) @ rng.standard_normal((r_true, 150))
    res = dashsvd(A, k=6, s=3, p_max=0, tol=0.0, seed=13)
    sv = np.linalg.svd(A, compute_uv=False)
    np.testing.assert_allclose(res.S[:r_true], sv[:r_true], rtol=1e-10)
    assert res.S[r_true] < 1e-6 * sv[0]
    Ur, _, Vtr = np.linalg.svd(A, full_matrices=False)
    assert np.max(metrics.principal_angles(res.U[:, :r_true], Ur[:, :r_true])) < 1e-7
    assert np.max(metrics.principal_angles(res.V[:, :r_true], Vtr[:r_true].T)) < 1e-7


def test_singular_values_never_exceed_true_prop2():
    A = _sparse(500, 200, 0.05, 6)
    sv = np.linalg.svd(A.toarray(), compute_uv=False)
    for p in range(5):
        r = dashsvd(A, 20, 10, p_max=p, tol=0.0, seed=14)
        assert np.all(r.S <= sv[:20] * (1 + 1e-12))


def test_per_pass_invariants_prop1_prop3():
    """Every pass: 0 <= alpha <= sigma_l(A)^2 / 2, alpha non-decreasing (Prop. 1, step 6)
    and sigma_i(A Q_in) <= sqrt(Shat_i + alpha) <= sigma_i(A) (Prop. 3)."""
    A = _sparse(600, 250, 0.04, 7)
    k, s = 15, 10
    l = k + s
    sv = np.linalg.svd(A.toarray(), compute_uv=False)
    r = dashsvd(A, k, s, p_max=8, tol=0.0, seed=15, keep_q=True)
    assert len(r.trace) == 8
    prev = 0.0
    for rec in r.trace:
        assert 0.0 <= rec.alpha_used <= sv[l - 1] ** 2 / 2 * (1 + 1e-12)
        assert rec.alpha_next >= rec.alpha_used
        assert rec.alpha_used >= prev
        prev = rec.alpha_used
        surrogate = np.sqrt(rec.S + rec.alpha_used)
        lower = np.linalg.svd(A @ rec.Q_in, compute_uv=False)
        assert np.all(lower <= surrogate * (1 + 1e-10))
        assert np.all(surrogate <= sv[:l] * (1 + 1e-10))
    assert r.trace[0].alpha_used == 0.0 and r.trace[1].alpha_used > 0.0


def _gap_case():
    """sigma_1..12 in [5, 10], then a gap to sigma_13..100 in [1, 2]: with l = 12
    the l-th Ritz value converges fast."""
    sv = np.r_[np.linspace(10, 5, 12), np.linspace(2.0, 1.0, 88)]
    return datagen.dense_with_spectrum(150, 100, sv, 3), sv


def test_shift_converges_to_half_sigma_l_squared():
    """Step 6's fixed point: once sqrt(Shat_l + alpha) has converged to sigma_l
    (Prop. 3's surrogate), alpha = (Shat_l + alpha) / 2 has the fixed point
    sigma_l^2 / 2, the top of Prop. 1's safe range; alpha approaches it from
    below without overshooting."""
    A, sv = _gap_case()
    r = dashsvd(A, 8, 4, p_max=20, tol=0.0, seed=2)
    target = sv[11] ** 2 / 2
    assert r.alpha <= target * (1 + 1e-12)
    assert abs(r.alpha - target) <= 1e-7 * target


def test_pve_stop_closed_form_full_width():
    """With l = n every surrogate is exact (Shat_i + alpha = sigma_i^2), so under
    reading R1 the test sees a zero change at j = 2 and stops there; taking
    step 7 literally mixes in the shift change and cannot stop at j = 2."""
    A = _sparse(120, 16, 0.3, 8)
    r0 = dashsvd(A, 10, 6, p_max=10, tol=1e-6, seed=16, alpha_prev_mode=0)
    assert r0.converged and r0.passes == 2
    sv = np.linalg.svd(A.toarray(), compute_uv=False)
    np.testing.assert_allclose(r0.trace[0].S + r0.trace[0].alpha_used, sv**2, rtol=1e-10)
    r1 = dashsvd(A, 10, 6, p_max=10, tol=1e-6, seed=16, alpha_prev_mode=1)
    assert r1.passes >= 3


def test_first_pass_never_stops_and_tol_monotone():
    A = _sparse(800, 300, 0.03, 9)
    passes = []
    for tol in [0.5, 1e-1, 1e-2, 1e-3, 1e-5]:
        r = dashsvd(A, 20, 10, p_max=30, tol=tol, seed=17)
        assert r.passes >= 2
        passes.append(r.passes)
    assert passes == sorted(passes)
    assert passes[-1] > passes[0]


def test_unshifted_mode_is_basic_power_iteration():
    """alpha = 0 gives span(Q) = span((A^T A)^p A^T Omega) (Alg. 1, m >= n form);
    the reference subspace is built here with QR instead of eigSVD."""
    A = _sparse(300, 120, 0.05, 10).toarray()
    k, s, p = 8, 4, 3
    l = k + s
    r = dashsvd(A, k, s, p_max=p, tol=0.0, seed=18, shift=False)
    Om = oracle.gaussian_block(18, 300, l)
    Q, _ = np.linalg.qr(A.T @ Om)
    for _ in range(p):
        Q, _ = np.linalg.qr(A.T @ (A @ Q))
    assert np.max(metrics.principal_angles(r.Q, Q)) < 1e-7
    r_shift = dashsvd(A, k, s, p_max=p, tol=0.0, seed=18)
    assert np.max(metrics.principal_angles(r_shift.Q, Q)) > 1e-6


def _theorem_case(seed, n=60, k=6, s=4, p=3):
    sigma = 1.0 / np.sqrt(np.arange(1, n + 1))
    A = datagen.dense_with_spectrum(n, n, sigma, seed)
    r = dashsvd(A, k, s, p_max=p, tol=0.0, seed=seed + 100)
    return A, sigma, r


def test_theorem1_bound_holds():
    """Theorem 1: ||A Q Q^T - A|| <= RHS with probability >= 1 - phi (here phi < 1e-3)."""
    n, k, s, p, j = 60, 6, 4, 3, 3
    l = k + s
    beta, gamma = 3.0, 2.5
    ph = metrics.phi(l, j, n, k, beta, gamma)
    assert ph < 1e-3
    held = 0
    for seed in range(50):
        A, sigma, r = _theorem_case(seed, n, k, s, p)
        alphas = [rec.alpha_used for rec in r.trace]
        rhs = metrics.theorem1_rhs(sigma, alphas, l, j, n, k, beta, gamma)
        err = np.linalg.norm(A @ r.Q @ r.Q.T - A, 2)
        held += err <= rhs
        # Corollary: the shifted bound never exceeds the unshifted one (strictly
        # smaller here because sigma_j > sigma_{k+1} and some alpha_c > 0)
        assert rhs < metrics.lemma6_rhs(sigma, p, l, j, n, k, beta, gamma)
    assert held >= 45


def test_shift_not_worse_statistically():
    """At equal p, the shifted run's eps_PVE is not worse than the unshifted one's
    (the paper shows this on Dense1/Dense2 and six datasets, Fig. 1); checked as
    a statistical property on 40 seeded cases per family."""
    fams = {
        "dense1": lambda sd: np.random.default_rng(sd).standard_normal((200, 200)),
        "dense2": lambda sd: datagen.dense_with_spectrum(200, 200, 1 / np.sqrt(np.arange(1, 201)), sd),
    }
    k, s, p = 10, 5, 2
    for name, mk in fams.items():
        ok = 0
        gains = []
        for sd in range(40):
            A = mk(sd)
            sv = np.linalg.svd(A, compute_uv=False)
            a = dashsvd(A, k, s, p_max=p, tol=0.0, seed=sd)
            b = dashsvd(A, k, s, p_max=p, tol=0.0, seed=sd, shift=False)
            ea = metrics.eps_pve(A, a.U, sv, k)
            eb = metrics.eps_pve(A, b.U, sv, k)
            ok += ea <= 1.05 * eb
            gains.append(eb / ea)
        assert ok >= 38, (name, ok)
        assert np.median(gains) > 1.0, name


def test_fixed_shift_mode_alg2_star():
    """Alg. 2* of Sec. 4: the shift is sigma_l(A A^T Q) / 2 from the first pass
    and then stays fixed; it is within Prop. 1's safe range, and at equal p the
    dynamic scheme is at least as accurate as the fixed one on most seeded
    Dense1 / Dense2 cases (the paper's Fig. 1 ordering, as a statistical
    property)."""
    fams = {
        "dense1": lambda sd: np.random.default_rng(100 + sd).standard_normal((200, 200)),
        "dense2": lambda sd: datagen.dense_with_spectrum(200, 200, 1 / np.sqrt(np.arange(1, 201)), 100 + sd),
    }
    k, s, p = 10, 5, 4
    l = k + s
    for name, mk in fams.items():
        ok = 0
        for sd in range(20):
            A = mk(sd)
            sv = np.linalg.svd(A, compute_uv=False)
            f = dashsvd(A, k, s, p_max=p, tol=0.0, seed=sd, shift="fixed")
            alphas = [t.alpha_used for t in f.trace]
            assert alphas[0] == 0.0 and len(set(alphas[1:])) == 1  # set once, then fixed
            assert alphas[1] == 0.5 * f.trace[0].S[l - 1]
            assert 0.0 < alphas[1] <= sv[l - 1] ** 2 / 2 * (1 + 1e-12)  # Prop. 1
            d = dashsvd(A, k, s, p_max=p, tol=0.0, seed=sd)
            ok += metrics.eps_pve(A, d.U, sv, k) <= 1.05 * metrics.eps_pve(A, f.U, sv, k)
        assert ok >= 17, (name, ok)


def test_config1_shape_runs_and_meets_tolerance():
    """The small workload (20000 x 10000 recipe at 1/10 scale): the run stops
    by the PVE test and the true eps_PVE is of the order of the tolerance."""
    A, prm = datagen.make_config(1, scale=0.1)
    As = A.to_scipy()
    r = dashsvd(As, prm["k"], prm["s"], p_max=prm["p_max"], tol=prm["tol"], seed=0x5EED)
    assert r.converged and 2 <= r.passes <= prm["p_max"]
    sv = np.linalg.svd(As.toarray(), compute_uv=False)
    assert metrics.eps_pve(As, r.U, sv, prm["k"]) < 10 * prm["tol"]
    assert metrics.eps_sigma(r.S, sv, prm["k"]) < 0.1


# ------------------------------------- accuracy control without the surrogate


def _eq19_stop_pass(A, k, s, tol, p_max, seed):
    """The first pass j >= 1 at which Eq. 19 holds, with sigma^(j) the singular
    values of A Q from a separate fixed-p run (Alg. 4, tol = 0) for each p = j."""
    sig = []
    for p in range(p_max + 1):
        r = dashsvd(A, k, s, p_max=p, tol=0.0, seed=seed)
        sig.append(np.linalg.svd(np.asarray(A @ r.Q), compute_uv=False))
    for j in range(1, p_max + 1):
        if np.max(np.abs(sig[j][:k] ** 2 - sig[j - 1][:k] ** 2)) / sig[j][k] ** 2 <= tol:
            return j
    return None


_DIRECT_CASES = {
    "dense2": lambda: datagen.dense_with_spectrum(200, 150, 1 / np.sqrt(np.arange(1, 151)), 7),
    "geometric": lambda: datagen.dense_with_spectrum(200, 150, 0.5 ** np.arange(150), 8),
    "config1": lambda: datagen.make_config(1, scale=0.05)[0].to_scipy(),
}


@pytest.mark.parametrize("case", sorted(_DIRECT_CASES))
def test_direct_pve_mode_stops_where_eq19_first_holds(case):
    """pve_mode="direct" (Table 4's control without the surrogate) stops at the
    first p whose fixed-p result satisfies Eq. 19 against the p - 1 result, and
    returns that fixed-p run's factors. On the fast-decaying spectrum p = 0 is
    already close, so the test can pass at j = 1 (sigma^(0) from step 2's basis)."""
    A = _DIRECT_CASES[case]()
    k, s, p_max, seed = 10, 5, 12, 3
    stops = []
    for tol in (0.5, 1e-1, 1e-2, 1e-3, 1e-4):
        d = dashsvd(A, k, s, p_max=p_max, tol=tol, seed=seed, pve_mode="direct")
        expect = _eq19_stop_pass(A, k, s, tol, p_max, seed)
        assert expect is not None and d.converged and d.passes == expect, (tol, d.passes, expect)
        f = dashsvd(A, k, s, p_max=d.passes, tol=0.0, seed=seed)
        assert np.array_equal(d.S, f.S) and np.array_equal(d.U, f.U) and np.array_equal(d.V, f.V)
        stops.append(d.passes)
    assert stops == sorted(stops)  # a tighter tolerance never stops earlier
    if case == "geometric":
        assert stops[0] == 1


def test_direct_pve_mode_only_changes_the_stop():
    """Without a stop test (tol = 0) both controls run the same iteration."""
    A = _DIRECT_CASES["config1"]()
    d = dashsvd(A, 12, 6, p_max=5, tol=0.0, seed=4, pve_mode="direct")
    r = dashsvd(A, 12, 6, p_max=5, tol=0.0, seed=4)
    assert d.passes == r.passes == 5 and not d.converged
    assert np.array_equal(d.S, r.S) and np.array_equal(d.U, r.U)
    assert [t.alpha_used for t in d.trace] == [t.alpha_used for t in r.trace]


def test_direct_pve_mode_needs_same_or_one_fewer_pass():
    """The paper's Table 4 observation: without the surrogate, N_p is the same
    or one smaller (here on the three seeded cases over five tolerances)."""
    for mk in _DIRECT_CASES.values():
        A = mk()
        for tol in (0.5, 1e-1, 1e-2, 1e-3, 1e-4):
            d = dashsvd(A, 10, 5, p_max=12, tol=tol, seed=3, pve_mode="direct")
            r = dashsvd(A, 10, 5, p_max=12, tol=tol, seed=3)
            assert r.passes - 1 <= d.passes <= r.passes, (tol, d.passes, r.passes)


def test_direct_pve_mode_rejects_bad_arguments():
    A = _DIRECT_CASES["config1"]()
    with pytest.raises(ValueError):
        dashsvd(A, 4, 2, p_max=2, tol=0.0, seed=1, pve_mode="exact")
    with pytest.raises(ValueError):
        dashsvd(A, 4, 2, p_max=2, tol=0.0, seed=1, pve_mode="direct", policy=lambda x: (1.0, -1.0))


# ------------------------------------------------------ planted mistakes


def _mutant_no_sqrt(C, eps=oracle.EPS64):
    U, S, V, null = eigsvd(C, eps)
    return U, S**2, V, null


def _mutant_ascending(C, eps=oracle.EPS64):
    U, S, V, null = eigsvd(C, eps)
    return U[:, ::-1], S[::-1], V[:, ::-1], null[::-1]


@pytest.mark.parametrize("mutant", [_mutant_no_sqrt, _mutant_ascending])
def test_pins_catch_planted_mistakes(monkeypatch, mutant):
    """Plant a mistake in the oracle's eigSVD and check that a pin fails."""
    import oracle.dashsvd_ref as ref

    A = _sparse(90, 14, 0.3, 3)
    Ur, Sr, Vtr = np.linalg.svd(A.toarray(), full_matrices=False)
    monkeypatch.setattr(ref, "eigsvd", mutant)
    r = ref.dashsvd(A, 9, 5, p_max=2, tol=0.0, seed=11)
    assert not np.allclose(r.S, Sr[:9], rtol=1e-6)


@pytest.mark.parametrize("mutant", ["unsquared", "pre_update_basis"])
def test_direct_pin_catches_planted_mistakes(monkeypatch, mutant):
    """Plant a mistake in the oracle's direct control (ratio on unsquared
    values; the test taken on the basis from before the pass) and check that the
    Eq. 19 pin disagrees for at least one tolerance."""
    import oracle.dashsvd_ref as ref

    A = _DIRECT_CASES["dense2"]()
    if mutant == "unsquared":
        monkeypatch.setattr(ref, "direct_pve_ratio",
                            lambda a, b, k: float(np.max(np.abs(a[:k] - b[:k])) / b[k]))
    else:
        real = ref.direct_pve_ratio
        hist = []

        def lagged(a, b, k):  # compares the pass before's values instead of this pass's
            hist.append(b)
            return real(hist[-3], hist[-2], k) if len(hist) >= 3 else np.inf

        monkeypatch.setattr(ref, "direct_pve_ratio", lagged)
    got, want = [], []
    for tol in (0.5, 1e-1, 1e-2, 1e-3, 1e-4):
        got.append(ref.dashsvd(A, 10, 5, p_max=12, tol=tol, seed=3, pve_mode="direct").passes)
    monkeypatch.undo()
    for tol in (0.5, 1e-1, 1e-2, 1e-3, 1e-4):
        want.append(_eq19_stop_pass(A, 10, 5, tol, 12, 3))
    assert got != want


@pytest.mark.parametrize("mutant", ["no_alpha_term", "no_half"])
def test_shift_pin_catches_planted_mistakes(monkeypatch, mutant):
    """Plant a mistake in the oracle's step 6 (the new shift without the old
    alpha term, or without the halving) and check that a pin fails."""
    import oracle.dashsvd_ref as ref

    if mutant == "no_alpha_term":
        monkeypatch.setattr(ref, "next_shift", lambda S_l, alpha, f=1.0: 0.5 * S_l if S_l > alpha else alpha)
    else:
        monkeypatch.setattr(ref, "next_shift", lambda S_l, alpha, f=1.0: S_l + alpha if S_l > alpha else alpha)
    A, sv = _gap_case()
    r = ref.dashsvd(A, 8, 4, p_max=20, tol=0.0, seed=2)
    target = sv[11] ** 2 / 2
    assert abs(r.alpha - target) > 1e-3 * target
