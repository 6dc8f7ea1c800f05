"""The precision form's FP64 eigensolver in isolation (dashsvd_eig_fp64):
FP32 Jacobi to FP32 rounding, then Ogita-Aishima refinement steps in FP64
against the FP64 Gram (Alg. 3 step 1 carried in FP64).

Reference: LAPACK's symmetric eigensolver (numpy.linalg.eigh) on the very
same FP64 matrix. A backward-stable FP64 eigensolver is within a small
multiple of eps64 * ||G|| of the exact eigenvalues, so both sides agree to
1e-12 * ||G|| when the refinement works; the FP32 Jacobi result alone (no
refinement step) is off by about eps32 * ||G|| and must fail that bound,
which shows that the FP64 accuracy comes from the refinement.

The Grams: an exact one (small-integer C, whose BF16x3 tensor-core Gram is
then exact in FP64, so the whole precision-form chain is checked), Grams of
dashSVD's shifted passes (eigenvalues graded like sigma^4), and matrices
with exactly repeated eigenvalues, where only the eigenvectors' subspace is
determined and is compared as such.
"""
import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ds():
    import torch

    assert torch.cuda.is_available()
    import paper_2404_09276_gb300 as mod

    return mod


@pytest.fixture(scope="module")
def h(ds):
    with ds.Handle() as hh:
        yield hh


def _check(ds, h, G, iters=3, clusters=()):
    import torch

    l = G.shape[0]
    Gd = torch.as_tensor(G).cuda()
    D, V = h.eig_fp64(Gd, l, iters)
    torch.cuda.synchronize()
    D, V = D.cpu().numpy(), V.cpu().numpy()
    ref, Vr = np.linalg.eigh(G)
    ref, Vr = ref[::-1], Vr[:, ::-1]
    nrm = np.linalg.norm(G, 2)
    err = np.max(np.abs(D - ref)) / nrm
    res = np.linalg.norm(G @ V - V * D, axis=0).max() / nrm
    orth = np.abs(V.T @ V - np.eye(l)).max()
    for lo, hi in clusters:  # exactly repeated eigenvalues: compare the subspace
        # sine of the largest principal angle, from the part of the computed
        # basis outside the reference subspace (arccos of the cosines cannot
        # resolve angles below about 1e-8)
        P, R = V[:, lo:hi], Vr[:, lo:hi]
        sin_max = np.linalg.norm(P - R @ (R.T @ P), 2)
        assert sin_max < 1e-10, sin_max
    return err, res, orth


def _shifted_pass_grams():
    A, _ = datagen.make_config(2, scale=0.01)  # 10 000 x 10 000 power-law graph
    r = oracle.dashsvd(A.to_scipy(), 100, 50, p_max=3, tol=0.0, seed=0x5EED, keep_q=True)
    As = A.to_scipy().astype(np.float64)
    At = As.T.tocsr()
    out = []
    for rec in r.trace[1:3]:
        Cm = At @ (As @ rec.Q_in) - rec.alpha_used * rec.Q_in
        out.append(Cm.T @ Cm)
    return out


@pytest.mark.parametrize("rows,l", [(64, 40), (300, 150), (600, 256)])
def test_exact_integer_gram_through_bf16x3(ds, h, rows, l):
    """C with integer entries in [-8, 8]: BF16 holds them exactly (C_lo = 0)
    and every FP32 product and chunk sum is an integer below 2^24, so the
    tensor-core Gram equals C^T C exactly; its FP64 eigenvalues then match
    LAPACK's to 1e-12 ||G||."""
    import torch

    rng = np.random.default_rng(rows + l)
    ld = ds.ld_for(l)
    Cm = np.zeros((rows, ld), dtype=np.float32)
    Cm[:, :l] = rng.integers(-8, 9, (rows, l))
    G64 = h.gram_bf16x3(torch.as_tensor(Cm).cuda(), l)
    torch.cuda.synchronize()
    G = G64.cpu().numpy()
    C64 = Cm[:, :l].astype(np.float64)
    np.testing.assert_array_equal(G, C64.T @ C64)
    err, res, orth = _check(ds, h, G)
    assert err < 1e-12 and res < 1e-12 and orth < 1e-12, (err, res, orth)


def test_shifted_pass_grams(ds, h):
    for G in _shifted_pass_grams():
        err, res, orth = _check(ds, h, G)
        assert err < 1e-12 and res < 1e-12 and orth < 1e-12, (err, res, orth)


@pytest.mark.parametrize("l", [40, 150])
def test_repeated_eigenvalues(ds, h, l):
    """Clusters of 6 and 4 equal eigenvalues above a spread tail: the
    refinement keeps the invariant subspaces (only re-orthogonalizing inside
    a cluster) and the eigenvalues reach FP64 accuracy."""
    rng = np.random.default_rng(l)
    Q, _ = np.linalg.qr(rng.standard_normal((l, l)))
    d = np.concatenate([np.full(6, 3.0), np.full(4, 2.5), np.linspace(2.0, 0.01, l - 10)])
    G = (Q * d) @ Q.T
    G = (G + G.T) / 2
    err, res, orth = _check(ds, h, G, clusters=[(0, 6), (6, 10)])
    assert err < 1e-12 and res < 1e-12 and orth < 1e-12, (err, res, orth)


def test_without_refinement_the_bound_fails(ds, h):
    """The same exact Gram with no refinement step: the FP32 Jacobi result is
    only FP32-accurate, far outside 1e-12 ||G|| (this is what the refinement buys)."""
    rng = np.random.default_rng(300 + 150)
    C64 = rng.integers(-8, 9, (300, 150)).astype(np.float64)
    G = C64.T @ C64
    err0, _, orth0 = _check(ds, h, G, iters=0)
    err3, _, _ = _check(ds, h, G, iters=3)
    assert err0 > 1e-9 and orth0 > 1e-9
    assert err3 < 1e-12
