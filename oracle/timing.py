"""Timed samples of the FP64 oracle for the benchmark's CPU baseline.

TEST INFRASTRUCTURE: run only by bench.py (its cpu_baseline leg and its
``--impl reference`` arm), as a separate process.

A sample is one power-iteration pass of dashSVD (Alg. 5 step 4: the two
sparse products, the shift, and eigSVD of the n x l result) on the full
matrix, timed with the oracle exactly as it stands. The number of passes a
whole run needs comes from the caller.

Usage: python -m oracle.timing MATRIX.npz k s reps [--full-run p_max tol seed]
prints one JSON line {"t_pass": [...], "threads": T, ...}.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np


def _load(path):
    import scipy.sparse as sp

    z = np.load(path)
    m, n = int(z["m"]), int(z["n"])
    return sp.csr_matrix((z["val"].astype(np.float64), z["colidx"], z["rowptr"]), shape=(m, n))


def time_pass(A, k: int, s: int, reps: int) -> list[float]:
    from .dashsvd_ref import eigsvd

    m, n = A.shape
    if m < n:
        A = A.T.tocsr()
        m, n = n, m
    At = A.T.tocsr()
    l = k + s
    Q, _ = np.linalg.qr(np.random.default_rng(0).standard_normal((n, l)))
    out = []
    for _ in range(reps):
        t0 = time.perf_counter()
        C = At @ (A @ Q) - 0.5 * Q
        Qn, _, _, _ = eigsvd(C)
        out.append(time.perf_counter() - t0)
    return out


def main(argv):
    path, k, s, reps = argv[0], int(argv[1]), int(argv[2]), int(argv[3])
    A = _load(path)
    res = {"t_pass": time_pass(A, k, s, reps), "threads": os.cpu_count()}
    if "--full-run" in argv:
        i = argv.index("--full-run")
        p_max, tol, seed = int(argv[i + 1]), float(argv[i + 2]), int(argv[i + 3])
        from .dashsvd_ref import dashsvd

        t0 = time.perf_counter()
        r = dashsvd(A, k, s, p_max=p_max, tol=tol, seed=seed)
        res["t_full"] = time.perf_counter() - t0
        res["passes"] = r.passes
    print(json.dumps(res))


if __name__ == "__main__":
    main(sys.argv[1:])
