"""Accuracy metrics of Sec. 4 on the GPU (dashsvd_metrics) against the FP64
oracle's (oracle/metrics.py) on the same U, S, V: eps_PVE, eps_res and
eps_sigma from A^T U, and eps_spec from the block power method on the
residual against the exact spectral norm of the dense residual."""
import numpy as np
import pytest

import datagen
from oracle import metrics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ds():
    import torch

    assert torch.cuda.is_available()
    import paper_2404_09276_gb300 as mod

    return mod


def _case(m=1500, n=800, seed=31):
    sv = 1.0 / np.sqrt(np.arange(1, n + 1))  # the Dense2 spectrum of Sec. 4
    A = datagen.dense_with_spectrum(m, n, sv, seed).astype(np.float32)
    return datagen.dense_as_csr(A), A.astype(np.float64)


def _t(x):
    import torch

    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float32), device="cuda")


@pytest.mark.parametrize("p,k", [(1, 20), (3, 20), (2, 10)])
def test_metrics_match_oracle(ds, p, k):
    Ac, A = _case()
    sigma = np.linalg.svd(A, compute_uv=False)
    Ad = ds.CsrDevice.from_host(Ac)
    with ds.Handle() as h:
        U, S, V, _ = h.run(Ad, k, 10, p, 0.0)
        got = h.metrics(Ad, U, S, V, sigma[: k + 1], spec_block=16, spec_iters=40)
    Uh, Sh, Vh = (x.cpu().numpy().astype(np.float64) for x in (U, S, V))
    want = {"eps_pve": metrics.eps_pve(A, Uh, sigma, k), "eps_res": metrics.eps_res(A, Uh, Sh, Vh, sigma, k),
            "eps_sigma": metrics.eps_sigma(Sh, sigma, k), "eps_spec": metrics.eps_spec(A, Uh, Sh, Vh, sigma, k)}
    # FP32 A^T U: about 1e-6 of sigma_1^2 in ||A^T u_i||^2, over sigma_{k+1}^2 ~ 1/20
    for name in ("eps_pve", "eps_res", "eps_sigma"):
        assert abs(got[name] - want[name]) <= 1e-3 * want[name] + 5e-5, (name, got[name], want[name])
    # the power estimate of ||A - U S V^T||_2 approaches it from below
    assert abs(got["eps_spec"] - want["eps_spec"]) <= 1e-4, (got["eps_spec"], want["eps_spec"])
    assert got["spec_norm"] <= (1 + 1e-5) * (want["eps_spec"] + 1) * sigma[k]


def test_metrics_of_exact_svd_are_rounding_level(ds):
    Ac, A = _case(seed=32)
    Ue, Se, Vte = np.linalg.svd(A, full_matrices=False)
    k = 16
    Ad = ds.CsrDevice.from_host(Ac)
    with ds.Handle() as h:
        got = h.metrics(Ad, _t(Ue[:, :k]), _t(Se[:k]), _t(Vte[:k].T), Se[: k + 1], spec_iters=40)
    assert got["eps_pve"] < 1e-4 and got["eps_res"] < 3e-5 and got["eps_sigma"] < 1e-6
    assert abs(got["eps_spec"]) < 1e-4


def test_metrics_without_spectral_estimate(ds):
    Ac, A = _case(seed=33)
    sigma = np.linalg.svd(A, compute_uv=False)
    Ad = ds.CsrDevice.from_host(Ac)
    with ds.Handle() as h:
        U, S, V, _ = h.run(Ad, 8, 8, 2, 0.0)
        got = h.metrics(Ad, U, S, V, sigma[:9], spec_iters=0)
    assert np.isnan(got["eps_spec"]) and np.isnan(got["spec_norm"])
    assert np.isfinite(got["eps_pve"])


def test_metrics_argument_checks(ds):
    Ac, A = _case(m=300, n=200, seed=34)
    sigma = np.linalg.svd(A, compute_uv=False)
    Ad = ds.CsrDevice.from_host(Ac)
    with ds.Handle() as h:
        U, S, V, _ = h.run(Ad, 8, 4, 1, 0.0)
        bad = sigma[:9].copy()
        bad[8] = 0.0
        for kw, sig in [({}, bad), ({"spec_block": 17}, sigma[:9]), ({"spec_iters": -1}, sigma[:9])]:
            with pytest.raises(ds.DashSvdError) as e:
                h.metrics(Ad, U, S, V, sig, **kw)
            assert e.value.status == ds.DASHSVD_EINVAL
        with pytest.raises(ValueError):
            h.metrics(Ad, U, S, V, sigma[:5])
