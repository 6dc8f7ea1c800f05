"""options.deterministic: the CSR of A^T from a stable counting sort (each row
of A^T lists its entries in increasing row order of A, exactly the CSR of the
transpose with sorted indices), a fixed SpMM variant, and so bitwise-equal
results from run to run; the fused pass product (an atomic scatter) is refused."""
import numpy as np
import pytest
import scipy.sparse as sp

import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ds():
    import torch

    assert torch.cuda.is_available()
    import paper_2404_09276_gb300 as mod

    return mod


def _single_column():
    rng = np.random.default_rng(4)
    A = sp.random(500, 1, density=0.3, random_state=rng, format="csr", dtype=np.float32)
    return datagen.Csr(500, 1, A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float32))


def _long_row():
    """One row of 30 000 entries among short ones (a hot column of A^T is a long run of equal keys)."""
    rng = np.random.default_rng(5)
    m, n = 40000, 3000
    A = sp.random(m, n, density=5e-4, random_state=rng, format="lil", dtype=np.float32)
    A[:, 17] = rng.standard_normal((m, 1)).astype(np.float32) * (rng.random((m, 1)) < 0.75)
    A = A.tocsr()
    A.sort_indices()
    return datagen.Csr(m, n, A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float32))


MATRICES = {
    "cfg1x0.1": lambda: datagen.make_config(1, scale=0.1)[0],
    "social": lambda: datagen.make_config(2, scale=0.003)[0],
    "termdoc": lambda: datagen.make_config(3, scale=0.01)[0],
    "hot_column": _long_row,
    "single_column": _single_column,
}


@pytest.mark.parametrize("name", list(MATRICES))
def test_stable_transpose_is_the_sorted_csr_of_the_transpose(ds, name):
    A = MATRICES[name]()
    with ds.Handle(deterministic=1) as h:
        At = h.csr_transpose(ds.CsrDevice.from_host(A))
        rp, ci, va = (x.cpu().numpy() for x in (At.rowptr, At.colidx, At.val))
    ref = A.to_scipy(np.float32).T.tocsr()
    ref.sort_indices()
    np.testing.assert_array_equal(rp, ref.indptr)
    np.testing.assert_array_equal(ci, ref.indices)
    np.testing.assert_array_equal(va, ref.data)


@pytest.mark.parametrize("form", [0, 1])
def test_runs_are_bitwise_equal(ds, form):
    import torch

    A, prm = datagen.make_config(2, scale=0.01)  # 10 000 x 10 000 power-law graph
    Ad = ds.CsrDevice.from_host(A)
    outs = []
    for _ in range(2):
        with ds.Handle(deterministic=1, form=form) as h:  # a fresh handle: setup rebuilt each time
            U, S, V, info = h.run(Ad, 20, 10, 6, 0.0)
            torch.cuda.synchronize()
            outs.append((U.clone(), S.clone(), V.clone(), info.passes, (info.spmm_variant & 0xFF)))
    (U1, S1, V1, p1, v1), (U2, S2, V2, p2, v2) = outs
    assert p1 == p2 == 6 and v1 == v2 == 5
    assert torch.equal(S1, S2) and torch.equal(U1, U2) and torch.equal(V1, V2)
    # and it is the same computation as the default mode, up to rounding
    with ds.Handle(form=form, spmm_variant=5) as h:
        _, S3, _, _ = h.run(Ad, 20, 10, 6, 0.0)
        torch.cuda.synchronize()
    assert torch.allclose(S1, S3, rtol=1e-4, atol=0)


def test_fused_product_refused(ds):
    import ctypes as C

    import torch

    A, _ = datagen.make_config(1, scale=0.1)
    Ad = ds.CsrDevice.from_host(A)
    with ds.Handle(deterministic=1, spmm_variant=10) as h:
        U = torch.empty((A.m, 5), device="cuda")
        S = torch.empty((5,), device="cuda")
        V = torch.empty((A.n, 5), device="cuda")
        st = ds.dashsvd_run(h.h, C.byref(Ad.struct()), 5, 5, 2, 0.0, U.data_ptr(), S.data_ptr(), V.data_ptr(),
                            None)
        assert st == ds.DASHSVD_EINVAL
