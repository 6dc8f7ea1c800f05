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


# (rows, l) cases: the last two need more row chunks than the fixed array holds
# partial blocks for (at l = 150 one chunk's partial block is 160 x 160 floats,
# 163 of them fit in 4 Mi floats, and 100 000 rows would be split into about 300
# chunks; at l = 256 three 128 x 128 blocks per chunk, 85 chunks fit, 30 000 rows
# would take about 100), so the entry point must use fewer, longer chunks
CASES = [(20011, 150), (5000, 64), (100_000, 150), (30_000, 256)]


@pytest.mark.parametrize("first,second", [(0, 1), (2, 3), (3, 2)])
def test_noalloc_gram_matches_handle_gram_twice(first, second):
    import torch

    assert torch.cuda.is_available()
    import paper_2404_09276_gb300 as ds

    stream = torch.cuda.current_stream()
    with ds.Handle(stream=stream) as h:
        for call, (rows, l) in enumerate([CASES[first], CASES[second]]):
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
            # both are FP32 chunk sums added in FP64: a chunk of K rows is within
            # (K + 2) 2^-24 |C|^T|C| of its exact sum; the longest chunks here have
            # under 1 200 rows (100 000 rows over at least 85 chunks)
            tol = (1200 + 2) * 2.0**-24
            assert np.all(np.abs(a - b) <= 2 * tol * bound + 1e-30)
            assert np.all(np.abs(a - C64.T @ C64) <= tol * bound + 1e-30)
            rel = np.abs(a - C64.T @ C64)[bound > 0] / bound[bound > 0]
            assert np.median(rel) < 1e-6
            np.testing.assert_array_equal(a, a.T)


def test_noalloc_rejects_oversized_l():
    import torch

    import paper_2404_09276_gb300 as ds

    x = torch.zeros((8, 264), dtype=torch.float32, device="cuda")
    g = torch.zeros((257, 257), dtype=torch.float32, device="cuda")
    st = ds.dashsvd_gram_noalloc(x.data_ptr(), 8, 257, 264, g.data_ptr(), 257, None)
    assert st == ds.DASHSVD_EINVAL
