"""The device check of a CSR's structure (dashsvd_csr_check), and that
dashsvd_run and the step-level products refuse a malformed CSR before any
product runs.

The malformed inputs with column ids outside [0, n) or out-of-order row
pointers go to dashsvd_csr_check only: it reads just the declared m + 1 row
pointers and nnz column ids and gathers nothing. dashsvd_run and the
step-level SpMM get only malformations under which every access of the
products would still stay inside the arrays (a first row pointer of 1: row 0
merely loses an entry), so a broken check could not make them read out of
bounds.
"""
import numpy as np
import pytest

import datagen

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


def _dev(ds, m, n, rowptr, colidx, val):
    import torch

    return ds.CsrDevice(m, n, torch.as_tensor(np.asarray(rowptr, dtype=np.int32)).cuda(),
                        torch.as_tensor(np.asarray(colidx, dtype=np.int32)).cuda(),
                        torch.as_tensor(np.asarray(val, dtype=np.float32)).cuda())


def _base():
    A, _ = datagen.make_config(2, scale=0.002)  # 2000 x 2000 power-law graph
    return A


def test_valid_matrices_pass(ds, h):
    A = _base()
    st, flags = h.csr_check(_dev(ds, A.m, A.n, A.rowptr, A.colidx, A.val))
    assert (st, flags) == (ds.DASHSVD_OK, 0)
    # empty rows everywhere but one, and an empty matrix
    st, flags = h.csr_check(_dev(ds, 5, 7, [0, 0, 0, 3, 3, 3], [0, 3, 6], [1, 2, 3]))
    assert (st, flags) == (ds.DASHSVD_OK, 0)
    st, flags = h.csr_check(_dev(ds, 4, 4, [0, 0, 0, 0, 0], [0], [0.0]))  # nnz taken from colidx: 1
    assert st == ds.DASHSVD_EINVAL and flags == ds.DASHSVD_CSR_BAD_LAST


@pytest.mark.parametrize("case", ["col_n", "col_neg", "col_huge", "first", "order", "last_small", "last_big",
                                  "col_and_order"])
def test_malformed_matrices_are_flagged(ds, h, case):
    A = _base()
    rp, ci = A.rowptr.copy(), A.colidx.copy()
    rng = np.random.default_rng(7)
    want = 0
    if case in ("col_n", "col_and_order"):
        ci[rng.integers(0, A.nnz)] = A.n
        want |= ds.DASHSVD_CSR_BAD_COL
    if case == "col_neg":
        ci[A.nnz - 1] = -1
        want |= ds.DASHSVD_CSR_BAD_COL
    if case == "col_huge":
        ci[0] = 2**31 - 1
        want |= ds.DASHSVD_CSR_BAD_COL
    if case == "first":
        rp[0] = 1
        want |= ds.DASHSVD_CSR_BAD_FIRST
    if case in ("order", "col_and_order"):
        i = int(np.argmax(np.diff(rp) > 2))  # a row with at least 3 entries
        rp[i + 1] = rp[i + 2] + 1  # rowptr[i + 1] > rowptr[i + 2]
        want |= ds.DASHSVD_CSR_BAD_ORDER
    if case == "last_small":
        rp[-1] = A.nnz - 1
        want |= ds.DASHSVD_CSR_BAD_LAST
    if case == "last_big":
        rp[-1] = A.nnz + 5
        want |= ds.DASHSVD_CSR_BAD_LAST
    st, flags = h.csr_check(_dev(ds, A.m, A.n, rp, ci, A.val))
    assert st == ds.DASHSVD_EINVAL
    assert flags == want


def test_run_and_step_products_refuse_before_computing(ds, h):
    """rowptr[0] = 1 on an otherwise valid CSR: every product would stay in
    bounds, but the structure is wrong, so nothing may run."""
    import ctypes as C

    import torch

    A = _base()
    rp = A.rowptr.copy()
    rp[0] = 1
    Ad = _dev(ds, A.m, A.n, rp, A.colidx, A.val)
    k, s = 10, 5
    U = torch.full((A.m, k), 7.0, device="cuda")
    S = torch.full((k,), 7.0, device="cuda")
    V = torch.full((A.n, k), 7.0, device="cuda")
    info = ds.dashsvd_info()
    st = ds.dashsvd_run(h.h, C.byref(Ad.struct()), k, s, 3, 1e-2, U.data_ptr(), S.data_ptr(), V.data_ptr(),
                        C.byref(info))
    assert st == ds.DASHSVD_EINVAL
    torch.cuda.synchronize()
    assert torch.all(U == 7.0) and torch.all(S == 7.0) and torch.all(V == 7.0)
    X = torch.zeros((A.n, 16), device="cuda")
    Y = torch.full((A.m, 16), 7.0, device="cuda")
    st = ds.dashsvd_spmm(h.h, C.byref(Ad.struct()), X.data_ptr(), 16, 15, Y.data_ptr(), 16, -1)
    assert st == ds.DASHSVD_EINVAL
    torch.cuda.synchronize()
    assert torch.all(Y == 7.0)
    # the same matrix with its structure repaired runs
    Ag = _dev(ds, A.m, A.n, A.rowptr, A.colidx, A.val)
    h.run(Ag, k, s, 3, 1e-2, U, S, V)
    torch.cuda.synchronize()
    assert torch.all(torch.isfinite(S)) and float(S[0]) > 0


def test_trust_csr_skips_the_step_level_check(ds):
    """With options.trust_csr = 1 the step-level product runs without the
    check (here on a valid CSR) and matches the checked call."""
    import torch

    A = _base()
    Ad = _dev(ds, A.m, A.n, A.rowptr, A.colidx, A.val)
    X = torch.randn((A.n, 16), device="cuda")
    with ds.Handle(trust_csr=1) as ht, ds.Handle() as hc:
        y1 = ht.spmm(Ad, X, 16, variant=1)
        y2 = hc.spmm(Ad, X, 16, variant=1)
        torch.cuda.synchronize()
    assert torch.equal(y1, y2)
