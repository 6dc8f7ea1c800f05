"""Host-side pieces of the benchmark (no GPU): the clock sampler against a
fake nvidia-smi, the roofline record, the DRAM traffic looked up from the
committed ncu summary only while the SpMM sources are unchanged, the launch
count, the choice of the reported form and the accuracy record against the
oracle (sigma errors, principal angles, spectral gap)."""
import os
import stat
import sys
import time
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

FAKE_SMI = r'''#!/usr/bin/env python3
import datetime, sys, time
ms = int(sys.argv[sys.argv.index("-lms") + 1])
reason = "Active" if "--id=1" in sys.argv else "Not Active"
while True:
    ts = datetime.datetime.now().strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    print(f"{ts}, 0, 1995, 2070, 700.0, 0x0, Not Active, Not Active, Not Active, {reason}", flush=True)
    time.sleep(ms / 1000)
'''


@pytest.fixture
def fake_smi(tmp_path, monkeypatch):
    p = tmp_path / "nvidia-smi"
    p.write_text(FAKE_SMI)
    p.chmod(p.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")


def test_clock_sampler_keeps_the_timed_window(fake_smi):
    c = bench.ClockSampler(0)
    time.sleep(0.25)
    c.mark()
    time.sleep(0.4)
    r = c.stop()
    assert r["window"] == "timed region" and 4 <= r["samples"] <= 12
    assert r["sm_mhz"] == 1995.0 and r["sm_max_mhz"] == 2070.0 and r["reasons"] == []


def test_clock_sampler_reports_power_cap(fake_smi):
    c = bench.ClockSampler(1)
    c.mark()
    time.sleep(0.2)
    assert bench.ClockSampler.stop(c)["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_nvidia_smi(monkeypatch, tmp_path):
    monkeypatch.setenv("PATH", str(tmp_path))
    c = bench.ClockSampler(0)
    c.mark()
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]


def _record(bwd_s=0.0029, var=7):
    per_run = {"gaussian": 0.0004, "spmm_fwd": 6 * 0.0013, "spmm_bwd": 6 * bwd_s, "gram": 0.0025, "eig": 0.01,
               "project": 0.003, "host_gap": 0.0003}
    groups = {"gaussian": 1, "spmm_fwd": 6, "spmm_bwd": 6, "gram": 7, "eig": 7, "project": 7, "host_gap": 6}
    return {"kernels_s": {"spmm_fwd": 0.0013, "spmm_bwd": bwd_s, "gram": 0.00035, "project": 0.00038, "eig": 0.003},
            "kernel_s_per_run": per_run, "kernel_launch_groups_per_run": groups,
            "profiled_run": {"variants": [5, var], "passes": 5},
            "bytes": {"spmm_fwd": 1.332e9, "spmm_bwd": 1.932e9}, "spmm": {"variants": [5, var]},
            "form": "precision"}


def test_roofline_of_the_dominant_spmm():
    """The dominant step is A^T Y - alpha Q (6 launch groups: 5 passes and the
    prologue's A^T Omega, which reads no Q): achieved = the compulsory bytes of
    those launches over their in-loop device time."""
    A = types.SimpleNamespace(m=1_000_000, n=1_000_000, nnz=15_000_000)
    pk = {"hbm_gbs": 6790.0, "source": "measured", "sm_max_mhz": 2070.0}
    r = bench._roofline(_record(), A, 150, pk)
    assert r["kernel"] == "spmm_bwd" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    total = 6 * 1.932e9 - 4 * 1_000_000 * 150
    assert abs(r["achieved"] - total / (6 * 0.0029) / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 6790.0) < 1e-12
    assert abs(r["frac_of_nominal"] - r["achieved"] / 7900.0) < 1e-12
    assert abs(r["gathered_gbs"] - 15e6 * 150 * 4 / 0.0029 / 1e9) < 1e-9
    assert abs(r["achieved_isolated"] - 1.932e9 / 0.0029 / 1e9) < 1e-9
    if r["traffic"] is not None:  # the committed summary matches the current SpMM sources
        assert abs(r["dram_gbs"] - r["traffic"] / 0.0029 / 1e9) < 1e-9


def test_traffic_needs_the_same_sources(monkeypatch):
    t = bench._traffic("spmm_bwd", 7)
    if t is None:
        pytest.skip("the SpMM sources changed since the committed ncu capture")
    assert t > 1.932e9  # more DRAM bytes than the compulsory ones: re-read gathers
    monkeypatch.setattr(bench, "_git_blob_sha1", lambda p: "0" * 40)
    assert bench._traffic("spmm_bwd", 7) is None
    assert bench._traffic("spmm_bwd", 3) is None


def test_launch_count_matches_the_committed_launch_list():
    """One steady-state run of the chosen form on the 1M graph (5 passes, A Q
    by variant 5 and A^T Y - alpha Q by variant 7, setup kept, the overlapped
    schedule) against the kernel count of the committed ncu launch list."""
    n = bench._launches_per_run("precision_learned", 5, 5, 7, setup_reused=True)
    eig = 19
    # the final stage: B's Gram, eigensolve, U and V, U's column norms (4 kernels)
    assert n == 1 + (1 + 2 + 2 + 2 + eig + 2) + 5 * (2 + 2 + 2 + eig + 2) + (2 + eig + 2 + 4)
    assert bench._launches_per_run("precision_learned", 5, 5, 7, setup_reused=False) == n + 13
    # the serial schedule: the fused pass product replaces the two products (2 + 2 launches) by 2
    serial = bench._launches_per_run("precision", 5, 5, 7, overlap=False)
    assert bench._launches_per_run("precision", 5, 5, 7, fused=True, overlap=False) == serial - 5 * 2


def _form(name, eps, value=1.0):
    return {"form": name, "accuracy": {"eps_pve": eps}, "value": value}


def test_chosen_form_falls_back_when_the_learned_stop_misses_tol():
    """The learned form ships while its true eps_PVE meets tol; otherwise the
    precision form with the plain shift rule; a form without a stored reference
    counts as meeting tol; when none meets tol, the learned form is reported."""
    forms = ["plain", "precision", "precision_learned"]
    res = {"plain": _form("plain", 1.1e-3), "precision": _form("precision", 4e-3),
           "precision_learned": _form("precision_learned", 2.8e-3)}
    assert bench._choose_form(res, forms, 1e-2)["form"] == "precision_learned"
    res["precision_learned"] = _form("precision_learned", 1.97e-2)
    assert bench._choose_form(res, forms, 1e-2)["form"] == "precision"
    res["precision"] = _form("precision", 1.2e-2)
    assert bench._choose_form(res, forms, 1e-2)["form"] == "plain"
    res["plain"] = _form("plain", 1.5e-2)
    assert bench._choose_form(res, forms, 1e-2)["form"] == "precision_learned"
    res["precision"] = _form("precision", None)
    assert bench._choose_form(res, forms, 1e-2)["form"] == "precision"
    # one form asked for: that form, whatever its accuracy
    assert bench._choose_form({"plain": _form("plain", 0.5)}, ["plain"], 1e-2)["form"] == "plain"
    # the boundary: eps == tol meets it
    assert bench._choose_form({"precision_learned": _form("precision_learned", 1e-2),
                               "precision": _form("precision", 1e-3)},
                              ["precision", "precision_learned"], 1e-2)["form"] == "precision_learned"


@pytest.mark.parametrize("theta", [0.0, 1e-3, 0.4, 1.2])
def test_subspace_angle_of_a_rotated_plane(theta):
    """span(e1, e2) against span(e1, cos t e2 + sin t e3), each given through a
    non-orthogonal basis: the largest principal angle is t."""
    import numpy as np

    n = 7
    X = np.zeros((n, 2))
    X[0, 0] = X[1, 1] = 1.0
    Y = np.zeros((n, 2))
    Y[0, 0] = 1.0
    Y[1, 1], Y[2, 1] = np.cos(theta), np.sin(theta)
    mix = np.array([[2.0, 1.0], [0.5, 3.0]])
    assert abs(bench._subspace_angle(X @ mix, Y @ mix.T) - theta) < 1e-7


def test_vs_oracle_errors_and_gap():
    """Relative sigma errors against the oracle's sigma, the principal angles of
    U_k and V_k, and the gap from the oracle's last pass (sqrt(Shat + alpha))."""
    import numpy as np

    from oracle.dashsvd_ref import PassRecord, Result

    rng = np.random.default_rng(5)
    m, n, k = 40, 30, 3
    U = np.linalg.qr(rng.standard_normal((m, k)))[0]
    V = np.linalg.qr(rng.standard_normal((n, k)))[0]
    S = np.array([4.0, 2.0, 1.0])
    last = PassRecord(3, 0.5, np.array([15.5, 3.5, 0.5, 0.14]), 1e-3, True, 0.5)
    ref = Result(U, S, V, 3, True, 0.5, False, [last])
    out = bench._vs_oracle((U, S * np.array([1.0, 1.01, 0.98]), V), ref, k)
    assert abs(out["sigma_rel_max"] - 0.02) < 1e-12
    assert abs(out["sigma_rel_median"] - 0.01) < 1e-12
    assert out["angle_U_rad"] < 1e-7 and out["angle_V_rad"] < 1e-7
    # estimates sqrt(16, 4, 1, 0.64) = (4, 2, 1, 0.8): gap_3 = (1 - 0.8) / 1
    assert abs(out["gap_k"] - 0.2) < 1e-12 and out["oracle_passes"] == 3
    # a column of U turned towards the complement by 0.3 rad
    W = np.linalg.qr(np.hstack([U, rng.standard_normal((m, 1))]))[0][:, k]
    U2 = U.copy()
    U2[:, 2] = np.cos(0.3) * U[:, 2] + np.sin(0.3) * W
    assert abs(bench._vs_oracle((U2, S, V), ref, k)["angle_U_rad"] - 0.3) < 1e-7
