"""Write the reference singular values of the 1M x 1M social-graph workload.

TEST INFRASTRUCTURE: calls only the FP64 oracle. The benchmark uses the stored
values for its post-hoc accuracy check: a timed run counts only if its true
per-vector error (Sec. 4) is at most the tolerance,
  eps_PVE = max_{i<=k} |sigma_i^2 - ||A^T u_i||^2| / sigma_{k+1}^2,
which needs sigma_1 .. sigma_{k+1} of the matrix.

The values come from the oracle's dashSVD (Alg. 5 in FP64) with a wide sketch
(k = 110, s = 90) and many fixed passes, far beyond what the timed k = 100 run
needs; the convergence of the last pass (the Prop. 3 surrogate sqrt(Shat_i +
alpha), compared between the last two passes) is recorded in the header.

Usage: python -m tests.golden.make_reference_sigma [passes]   (about 5 minutes on 8 cores)
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "social_graph_1m_sigma.txt")


def main(argv):
    sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
    import datagen
    import oracle

    passes = int(argv[0]) if argv else 30
    A, prm = datagen.make_config(2)
    t0 = time.perf_counter()
    r = oracle.dashsvd(A.to_scipy(), 110, 90, p_max=passes, tol=0.0, seed=0x5EED)
    dt = time.perf_counter() - t0
    a, b = r.trace[-2], r.trace[-1]
    s_prev = np.sqrt(np.maximum(a.S[:110] + a.alpha_used, 0.0))
    s_last = np.sqrt(np.maximum(b.S[:110] + b.alpha_used, 0.0))
    change = float(np.max(np.abs(s_last[:101] - s_prev[:101]) / s_last[:101]))
    with open(OUT, "w") as f:
        f.write("# sigma_1..sigma_110 of the social-graph workload (1M x 1M, nnz %d, matrix seed 1002)\n" % A.nnz)
        f.write("# written by: python -m tests.golden.make_reference_sigma %d\n" % passes)
        f.write("# FP64 oracle dashSVD, k=110 s=90, %d fixed passes, Omega seed 0x5EED, %.0f s\n" % (passes, dt))
        f.write("# last-pass relative change of sqrt(Shat_i + alpha), i <= 101: %.3e\n" % change)
        for v in r.S[:110]:
            f.write("%.17e\n" % v)
    print(OUT, change, dt)


if __name__ == "__main__":
    main(sys.argv[1:])
