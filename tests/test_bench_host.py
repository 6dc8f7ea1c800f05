"""Host-side pieces of the benchmark (no GPU): the clock sampler against a
fake nvidia-smi, the roofline record, and the DRAM traffic looked up from the
committed ncu summary only while the SpMM sources are unchanged."""
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
