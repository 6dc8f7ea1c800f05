"""Failure paths on the GPU without a GPU fault: a bounded device wait that
runs out reports DASHSVD_ETIMEOUT and leaves the context usable; a failed
workspace allocation reports DASHSVD_ENOMEM and leaves the handle usable."""
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


def _small(ds):
    A, prm = datagen.make_config(1, scale=0.05)
    return A, ds.CsrDevice.from_host(A)


def _check_run(ds, h, A, Ad):
    U, S, V, info = h.run(Ad, 8, 4, 2, 0.0)
    ref = oracle.dashsvd(A.to_scipy(), 8, 4, p_max=2, tol=0.0, seed=0x5EED)
    assert info.passes == 2
    np.testing.assert_allclose(S.cpu().numpy(), ref.S, rtol=1e-4)


def test_bounded_wait_runs_out_and_context_stays_usable(ds):
    A, Ad = _small(ds)
    with ds.Handle() as h:
        assert ds.dashsvd_selftest_bounded_wait(h.h, 1000) == ds.DASHSVD_ETIMEOUT
        assert ds.dashsvd_selftest_bounded_wait(h.h, 0) == ds.DASHSVD_EINVAL
        _check_run(ds, h, A, Ad)  # the same handle, the same context


@pytest.mark.parametrize("nth", [1, 3, 12])
def test_failed_allocation_leaves_the_handle_usable(ds, nth):
    A, Ad = _small(ds)
    with ds.Handle() as h:
        assert ds.dashsvd_selftest_fail_alloc(nth) == ds.DASHSVD_OK
        try:
            with pytest.raises(ds.DashSvdError) as e:
                h.run(Ad, 8, 4, 2, 0.0)
            assert e.value.status == ds.DASHSVD_ENOMEM
        finally:
            ds.dashsvd_selftest_fail_alloc(0)
        _check_run(ds, h, A, Ad)
