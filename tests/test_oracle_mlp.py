"""Pins of the learned form's network in the FP64 oracle (CPU only).

Each check compares against something other than the oracle's own formulas:
central finite differences, closed forms, a hand-worked example, Prop. 1's
safe-shift bound, and the plain-rule / unshifted special cases.
"""
import numpy as np
import pytest

import datagen
import oracle
from oracle import mlp_ref as M


def _rand_params(rng, scale=0.5):
    return rng.standard_normal(M.N_PARAMS) * scale


def test_param_count_and_layout():
    assert M.N_PARAMS == 16 * 64 + 64 + 64 * 2 + 2 == 1218
    w = np.arange(M.N_PARAMS, dtype=np.float64)
    W1, b1, W2, b2 = M.unpack(w)
    assert W1[0, 0] == 0 and W1[63, 15] == 1023 and b1[0] == 1024 and W2[0, 0] == 1088 and b2[1] == 1217
    assert np.array_equal(M.pack(W1, b1, W2, b2), w)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    w = _rand_params(rng)
    X = rng.uniform(-2, 2, size=(9, 16))
    T = np.c_[rng.uniform(0, 1, 9), rng.integers(0, 2, 9)]
    Mk = np.c_[rng.uniform(0.5, 2, 9), rng.uniform(0.5, 2, 9)]
    _, g = M.loss_and_grad(w, X, T, Mk)
    h = 1e-6
    fd = np.empty_like(w)
    for i in range(M.N_PARAMS):
        e = np.zeros_like(w)
        e[i] = h
        fd[i] = (M.loss_and_grad(w + e, X, T, Mk)[0] - M.loss_and_grad(w - e, X, T, Mk)[0]) / (2 * h)
    assert np.linalg.norm(g - fd) <= 1e-7 * np.linalg.norm(fd)
    assert np.max(np.abs(g - fd)) <= 1e-8


def test_zero_weights_give_biases():
    b1 = np.linspace(-1, 1, 64)
    b2 = np.array([0.3, -0.7])
    w = M.pack(np.zeros((64, 16)), b1, np.zeros((2, 64)), b2)
    X = np.random.default_rng(2).standard_normal((5, 16))
    H, O = M.forward(w, X)
    assert np.allclose(H, np.tanh(b1)[None, :], rtol=0, atol=0)
    assert np.allclose(O, b2[None, :], rtol=0, atol=0)


def test_gradient_vanishes_at_perfect_targets():
    rng = np.random.default_rng(3)
    w = _rand_params(rng)
    X = rng.standard_normal((7, 16))
    _, O = M.forward(w, X)
    T = 1.0 / (1.0 + np.exp(-O))  # targets equal to the predictions
    L, g = M.loss_and_grad(w, X, T, np.ones((7, 2)))
    assert np.max(np.abs(g)) < 1e-15
    # BCE at its minimum is the binary entropy of the target
    p = T[:, 1]
    assert np.isclose(L, np.mean(-(p * np.log(p) + (1 - p) * np.log(1 - p))), rtol=1e-12)


def test_adam_first_step_closed_form():
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    w0 = np.array([1.0, 1.0, 1.0, 1.0])
    w1, m, v = M.adam(w0, g, np.zeros(4), np.zeros(4), 1, lr=0.1)
    # bias-corrected moments of one step are g and g^2: the step is lr g / (|g| + eps)
    assert np.allclose(w0 - w1, 0.1 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_adam_fits_a_teacher_network():
    rng = np.random.default_rng(4)
    teacher = _rand_params(rng, 0.8)
    X = rng.uniform(-2, 2, size=(256, 16))
    _, O = M.forward(teacher, X)
    T = np.c_[1 / (1 + np.exp(-O[:, 0])), (O[:, 1] > 0).astype(float)]
    w = _rand_params(rng, 0.1)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    L0 = M.loss_and_grad(w, X, T, np.ones_like(T))[0]
    for t in range(1, 1501):
        L, g = M.loss_and_grad(w, X, T, np.ones_like(T))
        w, m, v = M.adam(w, g, m, v, t, lr=3e-3)
    assert L < 0.25 * L0


def test_features_hand_worked_example():
    # l = 4, k = 2, Shat = [4, 2, 1, 0.5], alpha = 0.5 (used in the pass)
    # T = Shat + alpha = [4.5, 2.5, 1.5, 1.0]; Shat_l = 0.5 is not above alpha,
    # so the plain rule keeps alpha: bound = 0.5
    x = M.features([4.0, 2.0, 1.0, 0.5], 0.5, ratio=1e-2, ratio_prev=1e-1, j=3, p_max=10, tol=1e-2, k=2)
    expect = [0.3, -0.5, -0.25, -0.5, 0.5 / 4.5, 2.5 / 4.5, 1.5 / 4.5, 1.0 / 4.5, 1.5 / 2.5, 1.0 / 1.5,
              0.5 / 4.5, -0.25, 0.5, 1.5 / 4.5, 1.0 / 2.0, (1.5 - 0.5) / (2.5 - 0.5)]
    # (k + l) / 2 = 3rd value for the middle feature: T_3 = 1.5
    assert np.allclose(x, expect, rtol=1e-15, atol=1e-15)


def test_features_are_scale_free():
    rng = np.random.default_rng(5)
    S = np.sort(rng.uniform(0, 10, 30))[::-1]
    a = 0.3 * S[-1]
    x1 = M.features(S, a, 0.05, 0.2, 4, 20, 1e-2, 20)
    x2 = M.features(7.5 * S, 7.5 * a, 0.05, 0.2, 4, 20, 1e-2, 20)
    assert np.allclose(x1, x2, rtol=1e-13, atol=1e-15)
    assert np.all(np.abs(x1) <= 4.0)


def _small_problem():
    A, _ = datagen.make_config(1, scale=0.05)
    return A.to_scipy(), 8, 4


def test_policy_f1_reproduces_plain_rule():
    A, k, s = _small_problem()
    ref = oracle.dashsvd(A, k, s, p_max=8, tol=1e-3, seed=0x5EED)
    r = oracle.dashsvd(A, k, s, p_max=8, tol=1e-3, seed=0x5EED, policy=lambda x: (1.0, -1.0))
    assert r.passes == ref.passes
    assert [t.alpha_used for t in r.trace] == [t.alpha_used for t in ref.trace]
    assert np.array_equal(r.S, ref.S)


def test_policy_f0_is_the_unshifted_method():
    A, k, s = _small_problem()
    ref = oracle.dashsvd(A, k, s, p_max=6, tol=0.0, seed=0x5EED, shift=False)
    r = oracle.dashsvd(A, k, s, p_max=6, tol=0.0, seed=0x5EED, policy=lambda x: (0.0, -1.0))
    assert all(t.alpha_used == 0.0 for t in r.trace)
    assert np.array_equal(r.S, ref.S)


@pytest.mark.parametrize("f", [0.25, 0.7, 1.0])
def test_learned_shifts_stay_in_the_safe_range(f):
    """Prop. 1: 0 <= alpha <= sigma_l(A)^2 / 2 at every pass, for any fraction f."""
    A, k, s = _small_problem()
    l = k + s
    sv = np.linalg.svd(A.toarray(), compute_uv=False)
    r = oracle.dashsvd(A, k, s, p_max=8, tol=0.0, seed=0x5EED, policy=lambda x: (f, -1.0))
    for t in r.trace:
        assert 0.0 <= t.alpha_used <= sv[l - 1] ** 2 / 2 * (1 + 1e-12)


def test_learned_stop_is_gated_by_the_soft_tolerance():
    A, k, s = _small_problem()
    tol = 1e-3
    plain = oracle.dashsvd(A, k, s, p_max=10, tol=1e-14, seed=0x5EED)
    ratios = [t.ratio for t in plain.trace]
    expect = next(j for j, r in enumerate(ratios, start=1) if j >= 2 and r <= 3 * tol)
    r = oracle.dashsvd(A, k, s, p_max=10, tol=tol, seed=0x5EED, policy=lambda x: (1.0, 1.0))
    assert r.passes == expect
