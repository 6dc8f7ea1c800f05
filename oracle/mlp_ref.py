"""The learned shift/stop network of the learned form, in FP64.

TEST INFRASTRUCTURE: used by the tests only (parity of the GPU inference,
gradient and optimizer kernels, and of learned dashSVD runs).

A 16 -> 64 (tanh) -> 2 network reads features of one power-iteration pass
(Alg. 5 steps 4-6: the new singular-value estimates Shat, the shift alpha used
in the pass and the PVE surrogate ratio) and proposes
  * the next shift as a fraction f = sigmoid(o_0) of the safe bound: the
    plain rule's value (Shat_l + alpha) / 2 when Shat_l > alpha, else alpha.
    Prop. 1 keeps any shift in [0, sigma_l^2 / 2] safe, and that bound is the
    largest shift the plain rule itself would take (Alg. 5 step 6);
  * an early stop when o_1 > 0, honoured only from the second pass on and
    while the surrogate ratio is at most 3 tol; the surrogate test of step 5
    still stops the run by itself.
With f = 1 and o_1 <= 0 the policy is exactly the plain rule.

Parameter vector (1218 values, the order the library loads): W1 (64 x 16,
row-major), b1 (64), W2 (2 x 64), b2 (2).

Training loss over a batch of B passes with targets T (B x 2) and weights M
(B x 2):
  L = (1/B) sum_b [ M_b0 (sigmoid(o_b0) - T_b0)^2
                    + M_b1 (softplus(o_b1) - T_b1 o_b1) ]
(the second term is the binary cross-entropy of sigmoid(o_b1) against T_b1).
The optimizer is Adam (Kingma and Ba, ICLR 2015) with bias correction.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT = 16, 64, 2
N_PARAMS = N_HID * N_IN + N_HID + N_OUT * N_HID + N_OUT  # 1218
FEATURE_CLIP = 4.0


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    if w.shape != (N_PARAMS,):
        raise ValueError("expected %d parameters" % N_PARAMS)
    i = 0
    W1 = w[i:i + N_HID * N_IN].reshape(N_HID, N_IN)
    i += N_HID * N_IN
    b1 = w[i:i + N_HID]
    i += N_HID
    W2 = w[i:i + N_OUT * N_HID].reshape(N_OUT, N_HID)
    i += N_OUT * N_HID
    b2 = w[i:i + N_OUT]
    return W1, b1, W2, b2


def pack(W1, b1, W2, b2):
    return np.concatenate([np.ravel(W1), np.ravel(b1), np.ravel(W2), np.ravel(b2)]).astype(np.float64)


def safe_bound(S, alpha):
    """The plain rule's next shift (Alg. 5 step 6); also the cap of a learned shift."""
    l = len(S)
    return 0.5 * (S[l - 1] + alpha) if S[l - 1] > alpha else alpha


def features(S, alpha, ratio, ratio_prev, j, p_max, tol, k):
    """Features of pass j. S: Shat (descending, l values); alpha: the shift used in
    the pass; ratio / ratio_prev: the PVE surrogate ratio of this pass and of the
    one before (the same value at j = 1). Shift-related quantities are the
    surrogates T_i = Shat_i + alpha of sigma_i^2 (Prop. 3), relative to T_1."""
    S = np.asarray(S, dtype=np.float64)
    l = len(S)
    a = float(alpha)
    T1, Tk, Tk1, Tl = S[0] + a, S[k - 1] + a, S[k] + a, S[l - 1] + a
    Tm = S[(k + l) // 2 - 1] + a
    bound = safe_bound(S, a)

    def lg(r):
        return np.log10(max(r, 1e-12)) / 4.0 if not np.isnan(r) else 0.0

    def div(x, y):
        return x / y if y > 0 else 0.0

    x = np.zeros(N_IN)
    x[0] = j / p_max if p_max > 0 else 0.0
    x[1] = lg(ratio)
    x[2] = lg(ratio_prev)
    x[3] = lg(tol)
    x[4] = div(a, T1)
    x[5] = div(Tk, T1)
    x[6] = div(Tk1, T1)
    x[7] = div(Tl, T1)
    x[8] = div(Tk1, Tk)
    x[9] = div(Tl, Tk1)
    x[10] = div(bound, T1)
    x[11] = x[1] - x[2]
    x[12] = k / l
    x[13] = div(Tm, T1)
    x[14] = div(S[k], S[k - 1])  # next-pass contraction (sigma_{k+1}^2 - a) / (sigma_k^2 - a)
    x[15] = div(Tk1 - bound, Tk - bound)  # the same with the plain rule's next shift
    x[~np.isfinite(x)] = 0.0
    return np.clip(x, -FEATURE_CLIP, FEATURE_CLIP)


def sigmoid(o):
    return 1.0 / (1.0 + np.exp(-o))


def forward(w, X):
    """Hidden activations H (B x 64) and outputs O (B x 2) for features X (B x 16)."""
    W1, b1, W2, b2 = unpack(w)
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    H = np.tanh(X @ W1.T + b1)
    return H, H @ W2.T + b2


def loss_and_grad(w, X, T, M):
    """Batch loss L and its gradient with respect to the parameter vector."""
    W1, b1, W2, b2 = unpack(w)
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    T = np.atleast_2d(np.asarray(T, dtype=np.float64))
    M = np.atleast_2d(np.asarray(M, dtype=np.float64))
    B = X.shape[0]
    H, O = forward(w, X)
    p0, p1 = sigmoid(O[:, 0]), sigmoid(O[:, 1])
    softplus = np.logaddexp(0.0, O[:, 1])
    L = np.sum(M[:, 0] * (p0 - T[:, 0]) ** 2 + M[:, 1] * (softplus - T[:, 1] * O[:, 1])) / B
    dO = np.empty_like(O)
    dO[:, 0] = M[:, 0] * 2.0 * (p0 - T[:, 0]) * p0 * (1.0 - p0) / B
    dO[:, 1] = M[:, 1] * (p1 - T[:, 1]) / B
    gW2 = dO.T @ H
    gb2 = dO.sum(axis=0)
    dZ = (dO @ W2) * (1.0 - H * H)
    gW1 = dZ.T @ X
    gb1 = dZ.sum(axis=0)
    return float(L), pack(gW1, gb1, gW2, gb2)


def adam(w, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns the new (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def policy_fp32(w):
    """The network as a pass policy in FP32 (the precision the GPU decides in):
    x -> (f, o_1)."""
    W1, b1, W2, b2 = (np.asarray(a, dtype=np.float32) for a in unpack(w))

    def pol(x):
        x = np.asarray(x, dtype=np.float32)
        h = np.tanh(W1 @ x + b1)
        o = W2 @ h + b2
        return float(1.0 / (1.0 + np.exp(-np.float64(o[0])))), float(o[1])

    return pol
