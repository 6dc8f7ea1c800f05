"""GPU parity of each hot-path step through the C ABI, against the FP64 oracle
or the plain FP64 definition of the step, on seeded inputs that span several
tiles and a ragged tail.

Tolerances follow from FP32 arithmetic: a length-K FP32 dot product is within
(K + 2) * 2^-24 * sum|a_i x_i| of the exact value (standard bound gamma_K), so
errors are measured against the matching absolute-value product.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import datagen
import oracle

pytestmark = pytest.mark.gpu

EPS32 = 2.0**-24


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


def _t(x):
    import torch

    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


def _np(x):
    import torch

    torch.cuda.synchronize()
    return x.cpu().numpy().astype(np.float64)


def _padded(X, ld, fill=np.nan):
    """Copy X into an (rows x ld) FP32 block whose padding columns hold `fill`."""
    out = np.full((X.shape[0], ld), fill, dtype=np.float32)
    out[:, : X.shape[1]] = X
    return out


def _mixed_matrix(seed=3):
    """Short rows, empty rows, and one 30000-long row (forces split rows)."""
    rng = np.random.default_rng(seed)
    m, n = 3000, 40000
    A = sp.random(m, n, density=4e-4, random_state=rng, format="lil", dtype=np.float32)
    A[17, :] = 0
    A[2999, :] = 0
    cols = rng.choice(n, 30000, replace=False)
    A[1234, cols] = rng.standard_normal(30000).astype(np.float32)
    A = A.tocsr()
    A.sort_indices()
    return datagen.Csr(m, n, A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float32))


_CACHE = {}


def _cached(name, make):
    # the matrices are generated once per session (read-only in every test)
    def get():
        if name not in _CACHE:
            _CACHE[name] = make()
        return _CACHE[name]

    return get


MATRICES = {
    "cfg1x0.1": _cached("cfg1x0.1", lambda: datagen.make_config(1, scale=0.1)[0]),
    "social": _cached("social", lambda: datagen.make_config(2, scale=0.003)[0]),
    "termdoc": _cached("termdoc", lambda: datagen.make_config(3, scale=0.01)[0]),
    "mixed": _cached("mixed", _mixed_matrix),
}


def test_gaussian_matches_oracle(ds, h):
    for l, rows, row0 in [(30, 1000, 0), (7, 333, 5), (150, 513, (1 << 32) + 9), (256, 64, 123456)]:
        Y = _np(h.gaussian(0x5EED, rows, l, row0))
        ref = oracle.gaussian_block(0x5EED, rows, l, row0)
        np.testing.assert_allclose(Y[:, :l], ref, rtol=1e-5, atol=2e-6)
        assert np.all(Y[:, l:] == 0.0)


@pytest.mark.parametrize("name", list(MATRICES))
def test_csr_transpose_exact(ds, h, name):
    A = MATRICES[name]()
    At = h.csr_transpose(ds.CsrDevice.from_host(A))
    ref = A.to_scipy(np.float32).T.tocsr()
    ref.sort_indices()
    rp = At.rowptr.cpu().numpy()
    ci = At.colidx.cpu().numpy()
    va = At.val.cpu().numpy()
    np.testing.assert_array_equal(rp, ref.indptr)
    for r in range(At.m):  # entries of a row come in no fixed order: compare sorted
        a, b = rp[r], rp[r + 1]
        o = np.argsort(ci[a:b], kind="stable")
        np.testing.assert_array_equal(ci[a:b][o], ref.indices[a:b])
        np.testing.assert_array_equal(va[a:b][o], ref.data[a:b])


def _spmm_check(A, X, Y, l):
    As = A.to_scipy(np.float64)
    ref = As @ X[:, :l].astype(np.float64)
    bound = abs(As) @ np.abs(X[:, :l].astype(np.float64))
    K = max(1, int(np.diff(A.rowptr).max()))
    err = np.abs(Y[:, :l] - ref)
    assert np.all(err <= (K + 2) * EPS32 * bound + 1e-30)
    med = np.median(err[bound > 0] / bound[bound > 0]) if np.any(bound > 0) else 0.0
    assert med < 1e-6


# 17, 19, 21, 22, 23: variants 1, 3, 5, 6, 7 with L2 eviction-priority hints
HINTED = [17, 19, 21, 22, 23]


@pytest.mark.parametrize("name", list(MATRICES))
@pytest.mark.parametrize("l", [1, 7, 30, 150, 160, 220, 256])
@pytest.mark.parametrize("variant", list(range(10)) + HINTED)
def test_spmm_matches_fp64(ds, h, name, l, variant):
    A = MATRICES[name]()
    rng = np.random.default_rng(l)
    ld = ds.ld_for(l)
    X = _padded(rng.standard_normal((A.n, l)).astype(np.float32), ld)  # NaN padding must be ignored
    Y = _np(h.spmm(ds.CsrDevice.from_host(A), _t(X), l, variant=variant))
    assert Y.shape == (A.m, ld)
    assert np.all(Y[:, l:] == 0.0)
    _spmm_check(A, X, Y, l)


@pytest.mark.parametrize("name", ["social", "mixed"])
@pytest.mark.parametrize("variant", list(range(10)) + HINTED)
def test_spmm_shift_matches_fp64(ds, h, name, variant):
    import torch

    A = MATRICES[name]()
    l = 30
    ld = ds.ld_for(l)
    rng = np.random.default_rng(1)
    Y = _padded(rng.standard_normal((A.m, l)).astype(np.float32), ld)
    Q = _padded(rng.standard_normal((A.n, l)).astype(np.float32), ld)
    alpha = 0.37
    ad = torch.tensor([alpha], dtype=torch.float64, device="cuda")
    At = h.csr_transpose(ds.CsrDevice.from_host(A))
    Z = _np(h.spmm_shift(At, _t(Y), l, ad, _t(Q), variant=variant))
    As = A.to_scipy(np.float64)
    ref = As.T @ Y[:, :l].astype(np.float64) - np.float32(alpha) * Q[:, :l].astype(np.float64)
    bound = abs(As.T) @ np.abs(Y[:, :l].astype(np.float64)) + alpha * np.abs(Q[:, :l])
    K = int(np.diff(At.rowptr.cpu().numpy()).max()) + 1
    assert np.all(np.abs(Z[:, :l] - ref) <= (K + 2) * EPS32 * bound + 1e-30)
    assert np.all(Z[:, l:] == 0.0)


@pytest.mark.parametrize("name", ["cfg1x0.1", "social", "mixed"])
@pytest.mark.parametrize("l", [7, 30, 150])
def test_spmm_fused_matches_fp64(ds, h, name, l):
    """Z = A^T (A Q) - alpha Q in one read of A: y_i in FP32 registers, then
    atomic FP32 adds into Z. Bound: both sums are FP32 sums of at most K terms
    of the absolute-value products."""
    import torch

    A = MATRICES[name]()
    ld = ds.ld_for(l)
    rng = np.random.default_rng(3)
    Q = _padded(rng.standard_normal((A.n, l)).astype(np.float32), ld)  # NaN padding must be ignored
    alpha = 0.37
    ad = torch.tensor([alpha], dtype=torch.float64, device="cuda")
    Z = _np(h.spmm_fused(ds.CsrDevice.from_host(A), _t(Q), l, ad))
    As = A.to_scipy(np.float64)
    Q64 = Q[:, :l].astype(np.float64)
    ref = As.T @ (As @ Q64) - np.float32(alpha) * Q64
    bound = abs(As.T) @ (abs(As) @ np.abs(Q64)) + alpha * np.abs(Q64)
    K = int(np.diff(A.rowptr).max()) + int(np.bincount(A.colidx, minlength=A.n).max()) + 4
    assert np.all(np.abs(Z[:, :l] - ref) <= K * EPS32 * bound + 1e-30)
    assert np.all(Z[:, l:] == 0.0)


@pytest.mark.parametrize("name", ["social", "mixed"])
@pytest.mark.parametrize("variant", [0, 1, 3, 5, 17, 21])
def test_spmm_bf16_matches_fp64(ds, h, name, variant):
    """BF16 dense operands (precision form): the products are exact in FP32 and
    accumulated in FP32; a BF16 output adds one rounding of 2^-9."""
    import torch

    A = MATRICES[name]()
    l = 150
    ld = ds.ld_for(l)
    rng = np.random.default_rng(2)
    X = torch.as_tensor(rng.standard_normal((A.n, ld)).astype(np.float32)).cuda()
    X[:, l:] = 0
    Xb = X.to(torch.bfloat16)
    Ad = ds.CsrDevice.from_host(A)
    Yb = torch.empty((A.m, ld), dtype=torch.bfloat16, device="cuda")
    Yf = torch.empty((A.m, ld), dtype=torch.float32, device="cuda")
    h.spmm_bf16(Ad, Xb, l, Yb, variant=variant)
    h.spmm_bf16(Ad, Xb, l, Yf, variant=variant)
    torch.cuda.synchronize()
    X64 = Xb.float().cpu().numpy().astype(np.float64)[:, :l]
    As = A.to_scipy(np.float64)
    ref = As @ X64
    bound = abs(As) @ np.abs(X64)
    K = int(np.diff(A.rowptr).max()) + 2
    yf = Yf.cpu().numpy().astype(np.float64)
    yb = Yb.float().cpu().numpy().astype(np.float64)
    assert np.all(np.abs(yf[:, :l] - ref) <= K * EPS32 * bound + 1e-30)
    assert np.all(np.abs(yb[:, :l] - ref) <= (K * EPS32 + 2.0**-8) * bound + 1e-30)
    assert np.all(yf[:, l:] == 0) and np.all(yb[:, l:] == 0)


def test_spmm_merge_path_matches_warp_per_row_closely(ds, h):
    """The two work splits add the same products in different groupings; both
    are within the FP32 bound of the exact result and close to each other."""
    A = MATRICES["mixed"]()
    l = 64
    X = np.random.default_rng(0).standard_normal((A.n, l)).astype(np.float32)
    Ad = ds.CsrDevice.from_host(A)
    y0 = _np(h.spmm(Ad, _t(X), l, variant=0))
    y1 = _np(h.spmm(Ad, _t(X), l, variant=1))
    y1b = _np(h.spmm(Ad, _t(X), l, variant=1))
    np.testing.assert_array_equal(y1, y1b)  # merge path is deterministic
    np.testing.assert_allclose(y0, y1, rtol=1e-4, atol=1e-4)
    for v in (6, 7):  # bulk-copy staging: same segments, one nonzero at a time
        y6 = _np(h.spmm(Ad, _t(X), l, variant=v))
        np.testing.assert_array_equal(y6, _np(h.spmm(Ad, _t(X), l, variant=v)))
        np.testing.assert_allclose(y6, y1, rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("rows,l", [(1, 1), (100, 30), (5000, 7), (20011, 150), (3000, 160), (70000, 64),
                                    (9001, 220), (3000, 256)])
def test_gram_matches_fp64(ds, h, rows, l):
    rng = np.random.default_rng(rows)
    ld = ds.ld_for(l)
    Cm = _padded((rng.standard_normal((rows, l)) * np.logspace(0, -2, l)).astype(np.float32), ld)
    G = _np(h.gram(_t(Cm), l))
    C64 = Cm[:, :l].astype(np.float64)
    ref = C64.T @ C64
    bound = np.abs(C64).T @ np.abs(C64)
    assert np.all(np.abs(G - ref) <= 2e-5 * bound + 1e-30)
    np.testing.assert_array_equal(G, G.T)


@pytest.mark.parametrize("rows,l", [(1, 1), (64, 16), (1000, 30), (20011, 150), (3000, 160), (70000, 64),
                                    (9001, 220), (3000, 256), (500000, 150)])
def test_gram_bf16x3_matches_fp64(ds, h, rows, l):
    """Tensor-core BF16x3 Gram: each product carries a relative error of about
    2^-16 (the dropped lo*lo term and the rounding of the split), plus FP32
    accumulation within a row chunk."""
    rng = np.random.default_rng(rows + 7)
    ld = ds.ld_for(l)
    Cm = _padded((rng.standard_normal((rows, l)) * np.logspace(0, -2, l)).astype(np.float32), ld)
    G = _np(h.gram_bf16x3(_t(Cm), l))
    C64 = Cm[:, :l].astype(np.float64)
    ref = C64.T @ C64
    bound = np.abs(C64).T @ np.abs(C64)
    err = np.abs(G - ref)
    assert np.all(err <= 4e-5 * bound + 1e-30), float(np.max(err / (bound + 1e-300)))
    np.testing.assert_allclose(G, G.T, rtol=1e-6, atol=1e-6 * np.abs(G).max())


@pytest.mark.parametrize("rows,l,cols,ldo", [(10, 4, 4, 4), (1000, 30, 30, 32), (12345, 150, 150, 152),
                                             (777, 150, 100, 100), (4097, 160, 37, 40), (5000, 220, 220, 224),
                                             (3000, 256, 200, 256)])
def test_project_matches_fp64(ds, h, rows, l, cols, ldo):
    import torch

    rng = np.random.default_rng(rows + l)
    ld = ds.ld_for(l)
    Cm = _padded(rng.standard_normal((rows, l)).astype(np.float32), ld)
    W = rng.standard_normal((l, cols)).astype(np.float32)
    out = torch.full((rows, ldo), float("nan"), dtype=torch.float32, device="cuda")
    Out = _np(h.project(_t(Cm), l, _t(W), cols, out=out))
    ref = Cm[:, :l].astype(np.float64) @ W.astype(np.float64)
    bound = np.abs(Cm[:, :l]).astype(np.float64) @ np.abs(W).astype(np.float64)
    assert np.all(np.abs(Out[:, :cols] - ref) <= (l + 2) * EPS32 * bound)
    assert np.all(Out[:, cols:] == 0.0)


@pytest.mark.parametrize("rows,l,cols,ldo", [(10, 4, 4, 4), (1000, 30, 30, 32), (12345, 150, 150, 152),
                                             (777, 150, 100, 100), (4097, 160, 37, 40), (5000, 220, 220, 224),
                                             (3000, 256, 200, 208), (300000, 150, 150, 152)])
def test_project_bf16x3_matches_fp64(ds, h, rows, l, cols, ldo):
    """Tensor-core BF16x3 projection: relative error about 2^-16 per product term
    plus FP32 accumulation over l terms."""
    import torch

    rng = np.random.default_rng(rows + l + 1)
    ld = ds.ld_for(l)
    Cm = _padded(rng.standard_normal((rows, l)).astype(np.float32), ld)
    W = rng.standard_normal((l, cols)).astype(np.float32)
    out = torch.full((rows, ldo), float("nan"), dtype=torch.float32, device="cuda")
    Out = _np(h.project_bf16x3(_t(Cm), l, _t(W), cols, out=out))
    ref = Cm[:, :l].astype(np.float64) @ W.astype(np.float64)
    bound = np.abs(Cm[:, :l]).astype(np.float64) @ np.abs(W).astype(np.float64)
    err = np.abs(Out[:, :cols] - ref)
    assert np.all(err <= (4e-5 + (l + 2) * EPS32) * bound), float(np.max(err / bound))
    assert np.all(Out[:, cols:] == 0.0)


@pytest.mark.parametrize("rows,l", [(500, 12), (4000, 30), (20000, 150), (3000, 160), (8000, 220)])
def test_eigsvd_precision_form_matches_oracle(ds, h, rows, l):
    """eigSVD in the precision form (BF16x3 Gram and projection, FP64-refined
    eig): the Gram's relative error about 2^-16 bounds the accuracy; S_i moves by
    about e / (2 S_i) for an absolute Gram error e ~ 2^-16 * S_1^2."""
    ld = ds.ld_for(l)
    spec = np.logspace(0, -1.5, l)
    Cm64 = datagen.dense_with_spectrum(rows, l, spec, seed=l + 3)
    Cm = _padded(Cm64.astype(np.float32), ld)
    U, S, V = (_np(x) for x in h.eigsvd(_t(Cm), l, form=ds.DASHSVD_FORM_PRECISION))
    Ur, Sr, Vr, _ = oracle.eigsvd(Cm[:, :l].astype(np.float64))
    assert np.all(np.abs(S - Sr) <= 4e-5 * Sr[0] ** 2 / Sr + 1e-6 * Sr)
    np.testing.assert_allclose(U[:, :l].T @ U[:, :l], np.eye(l), atol=5e-3)
    np.testing.assert_allclose((U[:, :l] * S) @ V.T, Cm[:, :l], atol=2e-4 * np.abs(Cm[:, :l]).max())


@pytest.mark.parametrize("rows,l", [(500, 12), (4000, 30), (20000, 150), (3000, 160), (300, 1), (8000, 220),
                                    (2000, 256), (900, 31)])
def test_eigsvd_matches_oracle(ds, h, rows, l):
    rng = np.random.default_rng(l)
    ld = ds.ld_for(l)
    spec = np.logspace(0, -1.5, l)
    Cm64 = datagen.dense_with_spectrum(rows, l, spec, seed=l)
    Cm = _padded(Cm64.astype(np.float32), ld)
    U, S, V = (_np(x) for x in h.eigsvd(_t(Cm), l))
    Ur, Sr, Vr, _ = oracle.eigsvd(Cm[:, :l].astype(np.float64))
    # eigSVD squares the conditioning: an absolute error e in the eigenvalues of
    # G = C^T C (e ~ 1e-5 * S_1^2 for FP32 sums over these row counts) moves
    # S_i = sqrt(D_i) by about e / (2 S_i)
    assert np.all(np.abs(S - Sr) <= 1e-5 * Sr[0] ** 2 / Sr + 2e-5 * Sr)
    # same ordering and sign convention: columns agree entry by entry up to FP32 eig accuracy
    gaps = np.minimum(np.abs(np.diff(np.r_[np.inf, Sr])), np.abs(np.diff(np.r_[Sr, -np.inf])))
    ok = gaps / Sr[0] > 1e-3
    np.testing.assert_allclose(V[:, ok], Vr[:, ok], atol=2e-3)
    np.testing.assert_allclose(U[:, :l].T @ U[:, :l], np.eye(l), atol=2e-3)
    np.testing.assert_allclose((U[:, :l] * S) @ V.T, Cm[:, :l], atol=1e-4 * np.abs(Cm[:, :l]).max())


def test_eigsvd_rank_deficient_null_columns(ds, h):
    rng = np.random.default_rng(9)
    rows, r, l = 2000, 5, 24
    Cm = (rng.standard_normal((rows, r)) @ rng.standard_normal((r, l))).astype(np.float32)
    U, S, V = (_np(x) for x in h.eigsvd(_t(_padded(Cm, ds.ld_for(l))), l))
    sv = np.linalg.svd(Cm.astype(np.float64), compute_uv=False)
    np.testing.assert_allclose(S[:r], sv[:r], rtol=1e-5)
    assert np.all(S[r:] < 1e-2 * S[0])
    np.testing.assert_allclose(U[:, :r].T @ U[:, :r], np.eye(r), atol=1e-5)
    # columns whose eigenvalue is at the FP32 noise level are either nulled or finite
    assert np.all(np.isfinite(U)) and np.all(U[:, r:l][:, S[r:] < 1e-4 * S[0]] == 0.0)
