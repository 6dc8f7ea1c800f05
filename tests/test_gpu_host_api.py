"""dashsvd_run_host: dashSVD with A and U, S, V in host memory (the call a
user without device buffers makes), against dashsvd_run on device copies of
the same matrix; with options.deterministic both are bitwise equal."""
import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("pinned", [True, False])
def test_run_host_matches_run(pinned):
    import torch

    assert torch.cuda.is_available()
    import paper_2404_09276_gb300 as ds

    A, prm = datagen.make_config(1, scale=0.1)  # 2000 x 1000
    k, s = prm["k"], prm["s"]
    Ad = ds.CsrDevice.from_host(A)
    with ds.Handle(deterministic=1) as h:
        U1, S1, V1, i1 = h.run(Ad, k, s, 4, 1e-2)
        torch.cuda.synchronize()
        U1, S1, V1 = U1.cpu(), S1.cpu(), V1.cpu()
        mk = (lambda t: t.pin_memory()) if pinned else (lambda t: t)
        U2 = mk(torch.full((A.m, k), np.nan, dtype=torch.float32))
        S2 = mk(torch.full((k,), np.nan, dtype=torch.float32))
        V2 = mk(torch.full((A.n, k), np.nan, dtype=torch.float32))
        for _ in range(2):  # the second call keeps the setup of the first
            i2 = h.run_host(A, k, s, 4, 1e-2, U2, S2, V2)
            assert i2.passes == i1.passes and i2.status == i1.status
            assert torch.equal(S1, S2) and torch.equal(U1, U2) and torch.equal(V1, V2)
        assert i2.setup_reused == 1


def test_run_host_rejects_bad_structure():
    """The host copy is checked like any device CSR (an in-bounds malformation)."""
    import ctypes as C

    import torch

    import paper_2404_09276_gb300 as ds

    A, prm = datagen.make_config(1, scale=0.1)
    rp = A.rowptr.copy()
    rp[0] = 1
    csr = ds.dashsvd_csr(A.m, A.n, A.nnz, rp.ctypes.data, A.colidx.ctypes.data, A.val.ctypes.data)
    U = torch.zeros((A.m, 5))
    S = torch.zeros((5,))
    V = torch.zeros((A.n, 5))
    with ds.Handle() as h:
        st = ds.dashsvd_run_host(h.h, C.byref(csr), 5, 5, 2, 0.0, U.data_ptr(), S.data_ptr(), V.data_ptr(), None)
    assert st == ds.DASHSVD_EINVAL
