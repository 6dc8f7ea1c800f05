"""Time one step of the dashSVD hot path on a seeded workload, for profiling.

Runs a single kernel family through the library's step-level entry points
(``Handle.spmm``, ``spmm_shift``, ``spmm_fused``, ``gram[_bf16x3]``,
``project[_bf16x3]``, ``eigsvd``) on the matrix of one of the seeded
workloads, with ``--warmup`` untimed launches and ``--reps`` launches timed by
CUDA events, and prints one JSON line (median milliseconds, algorithmic bytes,
GB/s). Under a profiler, the warm-up launches come first, so ``ncu -s <warmup>
-c <reps>`` selects the timed ones.

Usage:
    python microbench.py --config 2 --product bwd --variant 7
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--product", default="bwd",
                    choices=["fwd", "bwd", "fused", "gram", "gram_bf16x3", "project", "project_bf16x3", "eigsvd"])
    ap.add_argument("--variant", type=int, default=-1, help="SpMM variant (fwd / bwd); + 16: with L2 hints")
    ap.add_argument("--variants", type=str, default="",
                    help="comma-separated SpMM variants to time one after the other (overrides --variant)")
    ap.add_argument("--l", type=int, default=0, help="block width (default: the workload's k + s)")
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--flush", action="store_true", help="write 256 MB before each timed launch (cold L2)")
    a = ap.parse_args(argv)

    sys.path.insert(0, ROOT)
    import torch

    import datagen
    import paper_2404_09276_gb300 as ds

    A, prm = datagen.make_config(a.config, a.scale)
    l = a.l or prm["k"] + prm["s"]
    ld = ds.ld_for(l)
    h = ds.Handle(trust_csr=1)  # the structure is checked once below, not on every timed call
    Ad = ds.CsrDevice.from_host(A)
    st_chk, flags = h.csr_check(Ad)
    assert st_chk == ds.DASHSVD_OK, flags
    At = h.csr_transpose(Ad) if a.product == "bwd" else None
    g = torch.Generator(device="cuda").manual_seed(0)
    rows = A.m if a.product in ("gram", "gram_bf16x3", "project", "project_bf16x3", "eigsvd") else A.n
    Q = torch.randn((A.n, ld), device="cuda", generator=g)
    Q[:, l:] = 0
    Y = torch.randn((A.m, ld), device="cuda", generator=g)
    Y[:, l:] = 0
    Z = torch.empty((A.n, ld), device="cuda")
    C = torch.randn((rows, ld), device="cuda", generator=g)
    C[:, l:] = 0
    W = torch.randn((l, ld), device="cuda", generator=g)
    Out = torch.empty((rows, ld), device="cuda")
    alpha = torch.tensor([0.5], dtype=torch.float64, device="cuda")
    csr_bytes = 4 * (A.m + 1) + 8 * A.nnz
    variants = [int(v) for v in a.variants.split(",")] if a.variants else [a.variant]
    for var in variants:
        _time_one(a, h, ds, torch, A, Ad, At, l, ld, Q, Y, Z, C, W, Out, alpha, rows, csr_bytes, var)
    h.close()


def _time_one(a, h, ds, torch, A, Ad, At, l, ld, Q, Y, Z, C, W, Out, alpha, rows, csr_bytes, variant):
    if a.product == "fwd":
        fn, nbytes = (lambda: h.spmm(Ad, Q, l, out=Y, variant=variant)), csr_bytes + 4 * A.n * l + 4 * A.m * ld
    elif a.product == "bwd":
        fn = lambda: h.spmm_shift(At, Y, l, alpha, Q, out=Z, variant=variant)  # noqa: E731
        nbytes = csr_bytes + 4 * A.m * l + 4 * A.n * l + 4 * A.n * ld
    elif a.product == "fused":
        fn, nbytes = (lambda: h.spmm_fused(Ad, Q, l, alpha, out=Z)), csr_bytes + 8 * A.n * l + 4 * A.n * ld
    elif a.product in ("gram", "gram_bf16x3"):
        f = h.gram if a.product == "gram" else h.gram_bf16x3
        fn, nbytes = (lambda: f(C, l)), 4 * rows * l
    elif a.product in ("project", "project_bf16x3"):
        f = h.project if a.product == "project" else h.project_bf16x3
        fn, nbytes = (lambda: f(C, l, W, l, out=Out, ldo=ld)), 4 * rows * l + 4 * rows * ld
    else:
        fn, nbytes = (lambda: h.eigsvd(C, l, form=ds.DASHSVD_FORM_PRECISION)), 4 * rows * l * 2
    flush = torch.empty(64 * 1024 * 1024, device="cuda") if a.flush else None
    st = torch.cuda.current_stream()
    for _ in range(a.warmup):
        fn()
    torch.cuda.synchronize()
    ts = []
    for i in range(a.reps):
        if flush is not None:
            flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = float(np.median(ts))
    print(json.dumps({"config": a.config, "scale": a.scale, "product": a.product, "variant": variant, "l": l,
                      "m": A.m, "n": A.n, "nnz": A.nnz, "ms": ms, "bytes": nbytes, "gbs": nbytes / ms / 1e6}),
          flush=True)


if __name__ == "__main__":
    main()
