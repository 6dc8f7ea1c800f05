"""The allocation-free Gram entry point (dashsvd_gram_noalloc) against the
handle-based one (dashsvd_gram), through the C ABI.

Callers that cannot allocate device memory (graph capture, hosts whose own
allocator owns the GPU) use dashsvd_gram_noalloc, whose scratch is one fixed
device array inside the library. This file is collected last so that a run
stopping at the first failure has already run every other test; it passes on
its own in a fresh process as well.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_gram_matches_handle_gram_twice():
    import torch

    assert torch.cuda.is_available()
    import paper_2404_09276_gb300 as ds

    stream = torch.cuda.current_stream()
    with ds.Handle(stream=stream) as h:
        for call, (rows, l) in enumerate([(20011, 150), (5000, 64)]):
            rng = np.random.default_rng(100 + call)
            ld = ds.ld_for(l)
            Cm = np.zeros((rows, ld), dtype=np.float32)
            Cm[:, :l] = rng.standard_normal((rows, l)) * np.logspace(0, -2, l)
            Ct = torch.as_tensor(Cm).cuda()
            G_ref = h.gram(Ct, l)
            G_na = torch.full((l, l), float("nan"), dtype=torch.float32, device="cuda")
            st = ds.dashsvd_gram_noalloc(Ct.data_ptr(), rows, l, Ct.stride(0), G_na.data_ptr(), G_na.stride(0),
                                         C.c_void_p(stream.cuda_stream))
            assert st == ds.DASHSVD_OK, ds.dashsvd_status_string(st)
            torch.cuda.synchronize()
            a = G_na.cpu().numpy().astype(np.float64)
            b = G_ref.cpu().numpy().astype(np.float64)
            C64 = Cm[:, :l].astype(np.float64)
            bound = np.abs(C64).T @ np.abs(C64)
            # both are FP32 chunk sums added in FP64: each within 2e-5 |C|^T|C| of the exact G
            assert np.all(np.abs(a - b) <= 4e-5 * bound + 1e-30)
            assert np.all(np.abs(a - C64.T @ C64) <= 2e-5 * bound + 1e-30)
            np.testing.assert_array_equal(a, a.T)


def test_noalloc_rejects_oversized_l():
    import torch

    import paper_2404_09276_gb300 as ds

    x = torch.zeros((8, 264), dtype=torch.float32, device="cuda")
    g = torch.zeros((257, 257), dtype=torch.float32, device="cuda")
    st = ds.dashsvd_gram_noalloc(x.data_ptr(), 8, 257, 264, g.data_ptr(), 257, None)
    assert st == ds.DASHSVD_EINVAL
