"""Write the reference singular values of the benchmark workloads.

TEST INFRASTRUCTURE: calls only the FP64 oracle. The stored values are the
reference for the post-hoc accuracy checks: a timed run counts only if its
true per-vector error (Sec. 4) is at most the tolerance,
  eps_PVE = max_{i<=k} |sigma_i^2 - ||A^T u_i||^2| / sigma_{k+1}^2,
which needs sigma_1 .. sigma_{k+1} of the matrix; the variance study of App. B
(Fig. 11) and the Table 4 comparison score their runs against them too.

The values come from the oracle's dashSVD (Alg. 5 in FP64) with a sketch much
wider than the timed runs use and many fixed passes; the convergence of the
last pass (the Prop. 3 surrogate sqrt(Shat_i + alpha), compared between the
last two passes) is recorded in each file's header.

Usage: python -m tests.golden.make_reference_sigma [name ...]
  social_graph_1m     1M x 1M social graph (k = 110, s = 90, 30 passes; about 7 minutes on 8 cores)
  social_graph_100k   the same recipe at 100k x 100k (the Fig. 11 stand-in; about 1 minute)
  term_document_500k  500k x 100k term-document matrix (k = 110, s = 90, 30 passes)
  recommender_2m      2M x 200k recommender matrix (k = 210, s = 90, 25 passes; about 25 minutes on 8 cores)
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

# name: (config, scale, k, s, passes, values kept)
JOBS = {
    "social_graph_1m": (2, 1.0, 110, 90, 30, 110),
    "social_graph_100k": (2, 0.1, 110, 90, 30, 110),
    "term_document_500k": (3, 1.0, 110, 90, 30, 110),
    "recommender_2m": (5, 1.0, 210, 90, 25, 210),
}


def path(name: str) -> str:
    return os.path.join(HERE, f"{name}_sigma.txt")


def write(name: str) -> None:
    sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
    import datagen
    import oracle

    cfg, scale, k, s, passes, keep = JOBS[name]
    A, _ = datagen.make_config(cfg, scale=scale)
    t0 = time.perf_counter()
    r = oracle.dashsvd(A.to_scipy(), k, s, p_max=passes, tol=0.0, seed=0x5EED)
    dt = time.perf_counter() - t0
    a, b = r.trace[-2], r.trace[-1]
    s_prev = np.sqrt(np.maximum(a.S[:k] + a.alpha_used, 0.0))
    s_last = np.sqrt(np.maximum(b.S[:k] + b.alpha_used, 0.0))
    kk = min(k, keep)
    change = float(np.max(np.abs(s_last[:kk] - s_prev[:kk]) / s_last[:kk]))
    with open(path(name), "w") as f:
        f.write(f"# sigma_1..sigma_{keep} of workload {cfg} at scale {scale:g} ({A.m} x {A.n}, nnz {A.nnz}, "
                f"matrix seed {1000 + cfg})\n")
        f.write(f"# written by: python -m tests.golden.make_reference_sigma {name}\n")
        f.write(f"# FP64 oracle dashSVD, k={k} s={s}, {passes} fixed passes, Omega seed 0x5EED, {dt:.0f} s\n")
        f.write(f"# last-pass relative change of sqrt(Shat_i + alpha), i <= {kk}: {change:.3e}\n")
        for v in r.S[:keep]:
            f.write("%.17e\n" % v)
    print(path(name), change, dt, flush=True)


def main(argv):
    for name in argv or ["social_graph_1m"]:
        write(name)


if __name__ == "__main__":
    main(sys.argv[1:])
