"""Training of the learned form's shift/stop network, on the GPU.

The network (16 -> 64 tanh -> 2; see include/dashsvd.h, "learned form") is
trained on traces that the library itself produces on seeded matrices of the
training family (``datagen.training_matrix``), with the library's own feature,
loss-gradient and Adam kernels. Labels come from full runs:

* stop head: for each pass j of a plain-rule trace at which a learned stop is
  allowed (j >= 2, surrogate ratio <= 3 tol), label 1 when stopping there
  would already meet the tolerance with a margin: the true PVE error of the
  run stopped at pass j (Sec. 4: max_i |sigma_i^2 - ||A^T u_i||^2| /
  sigma_{k+1}^2, with reference sigma from a long, wide run) is at most tol / 2.
  Wrong stops weigh three times as much as missed ones;
* shift head: the fraction f in {0.5, 0.75, 1} of the plain rule's shift whose
  run stops after the fewest passes with the true error within tol (ties go
  to the larger f), as the target for every pass of that matrix.

Validation runs both the plain rule and the trained network on held-out
matrices (``datagen.VAL_SEED0`` onwards). A learned run fails when its true
PVE error exceeds tol on a matrix where the plain rule's run meets it; with
any failure the plain rule is what ships (the weights file says
``ship: plain``).

Usage (on a GPU):
    python -m paper_2404_09276_gb300.learn --train 240 --val 60 --out paper_2404_09276_gb300/mlp_shift_stop.txt
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
DEFAULT_WEIGHTS = os.path.join(HERE, "mlp_shift_stop.txt")
TOL = 1e-2
P_MAX = 20
FRACTIONS = (0.5, 0.75, 1.0)


def load_weights(path: str = DEFAULT_WEIGHTS):
    """(weights as float32 array, ship flag) from a weights file; (None, False)
    when there is none. ship is True only when validation had no failure."""
    if not os.path.exists(path):
        return None, False
    ship = False
    vals = []
    with open(path) as f:
        for line in f:
            if line.startswith("#"):
                if line.strip().startswith("# ship:"):
                    ship = line.split(":", 1)[1].strip() == "learned"
                continue
            if line.strip():
                vals.append(float(line))
    w = np.asarray(vals, dtype=np.float32)
    return (w if w.size == 1218 else None), ship


def _const_net(o0, o1):
    w = np.zeros(1218, dtype=np.float32)
    w[-2], w[-1] = o0, o1
    return w


def _logit(f):
    return 40.0 if f >= 1.0 else float(np.log(f / (1.0 - f)))


class _Problem:
    """One seeded matrix on the device, with its transposed CSR and reference sigma."""

    def __init__(self, ds, seed):
        import datagen

        self.A, prm = datagen.training_matrix(seed)
        self.k, self.s = prm["k"], prm["s"]
        self.l = self.k + self.s
        self.Ad = ds.CsrDevice.from_host(self.A)
        self.h = ds.Handle(form=ds.DASHSVD_FORM_PRECISION)
        self.At = self.h.csr_transpose(self.Ad)
        self.handles = {}
        # reference sigma_1..sigma_{k+1}: the plain FP32 form, wider sketch, many passes
        kr = self.k + 1
        sr = min(self.A.n - kr, max(self.s, 60))
        with ds.Handle() as hr:
            _, S, _, _ = hr.run(self.Ad, kr, sr, 25, 0.0)
        self.sigma = S.double().cpu().numpy()

    def eps_pve(self, U):
        import torch

        Up = torch.zeros((U.shape[0], (self.k + 3) // 4 * 4), dtype=torch.float32, device=U.device)
        Up[:, : self.k] = U
        Y = self.h.spmm(self.At, Up, self.k)[:, : self.k]
        cap = (Y.double() ** 2).sum(0).cpu().numpy()
        return float(np.max(np.abs(self.sigma[: self.k] ** 2 - cap)) / self.sigma[self.k] ** 2)

    def run(self, ds, p, tol, weights=None, trace=False):
        import torch

        key = (weights is not None, trace)
        if key not in self.handles:
            self.handles[key] = ds.Handle(form=ds.DASHSVD_FORM_PRECISION, learned=1 if weights is not None else 0,
                                          record_trace=1 if trace else 0)
        h = self.handles[key]
        if weights is not None:
            h.load_mlp(weights)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        U, S, V, info = h.run(self.Ad, self.k, self.s, p, tol)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        tr = h.trace() if trace else None
        return U, info, tr, dt

    def close(self):
        for h in self.handles.values():
            h.close()
        self.h.close()


def collect(ds, seed):
    """Trace records, stop targets/weights and the shift target of one matrix."""
    pr = _Problem(ds, seed)
    try:
        _, _, tr, _ = pr.run(ds, 14, 1e-14, trace=True)
        rec = np.array([[j, a, r, an, sw, *Sh] for j, a, r, an, sw, Sh in tr])
        n = rec.shape[0]
        T = np.zeros((n, 2))
        W = np.zeros((n, 2))
        for i in range(n):
            j, ratio = int(rec[i, 0]), rec[i, 2]
            if j >= 2 and ratio <= 3 * TOL:
                U, _, _, _ = pr.run(ds, j, 0.0)
                good = pr.eps_pve(U) <= 0.5 * TOL
                T[i, 1] = 1.0 if good else 0.0
                W[i, 1] = 1.0 if good else 3.0
        best = None
        for f in FRACTIONS:
            U, info, _, _ = pr.run(ds, P_MAX, TOL, weights=_const_net(_logit(f), -40.0))
            cost = info.passes + (0 if pr.eps_pve(U) <= TOL else 100)
            if best is None or cost <= best[0]:
                best = (cost, f)
        T[:, 0] = best[1]
        W[:, 0] = 1.0
        return rec, T, W, pr.l, pr.k
    finally:
        pr.close()


def compare(ds, seeds, weights):
    """Plain rule vs the network on each matrix: passes, wall seconds and the
    true PVE error of both runs (precision form, tol = TOL, p_max = P_MAX)."""
    rows = []
    for sd in seeds:
        pr = _Problem(ds, sd)
        try:
            pr.run(ds, P_MAX, TOL)  # warm-up (autotuning, graph capture)
            pr.run(ds, P_MAX, TOL, weights=weights)
            U, ip, _, tp = pr.run(ds, P_MAX, TOL)
            ep = pr.eps_pve(U)
            U, il, _, tl = pr.run(ds, P_MAX, TOL, weights=weights)
            el = pr.eps_pve(U)
            rows.append(dict(seed=sd, plain_passes=ip.passes, learned_passes=il.passes, plain_s=tp, learned_s=tl,
                             plain_eps=ep, learned_eps=el))
        finally:
            pr.close()
    return rows


def summarize(rows):
    """A learned run fails when its true PVE error exceeds tol on a matrix where
    the plain rule's run meets it (the plain rule's own misses are the
    surrogate test's, and are counted separately)."""
    fails = [r for r in rows if r["learned_eps"] > TOL and r["plain_eps"] <= TOL]
    return dict(n=len(rows), plain_passes=float(np.mean([r["plain_passes"] for r in rows])),
                learned_passes=float(np.mean([r["learned_passes"] for r in rows])),
                plain_s=float(np.sum([r["plain_s"] for r in rows])),
                learned_s=float(np.sum([r["learned_s"] for r in rows])),
                failures=len(fails), fail_seeds=[(r["seed"], round(r["learned_eps"], 4)) for r in fails],
                plain_failures=sum(r["plain_eps"] > TOL for r in rows),
                both_over=sum(r["plain_eps"] > TOL and r["learned_eps"] > TOL for r in rows))


def train(ds, X, T, W, steps=4000, lr=3e-3, seed=0):
    import torch

    rng = np.random.default_rng(seed)
    w0 = np.concatenate([rng.standard_normal(64 * 16) * 0.25, np.zeros(64), rng.standard_normal(128) * 0.1,
                         np.array([3.0, -3.0])]).astype(np.float32)
    Wd = torch.as_tensor(w0, device="cuda")
    m, v = torch.zeros_like(Wd), torch.zeros_like(Wd)
    Xd = torch.as_tensor(X, dtype=torch.float32, device="cuda")
    Td = torch.as_tensor(T, dtype=torch.float32, device="cuda")
    Md = torch.as_tensor(W, dtype=torch.float32, device="cuda")
    h = ds.Handle()
    grad = torch.empty_like(Wd)
    loss = torch.empty(1, device="cuda")
    losses = []
    for step in range(1, steps + 1):
        h.mlp_loss_grad(Wd, Xd, Td, Md, grad, loss)
        h.mlp_adam(Wd, grad, m, v, step, lr)
        if step == 1 or step % 500 == 0:
            losses.append(float(loss.item()))
    h.close()
    return Wd.cpu().numpy(), losses


def main(argv=None):
    import torch

    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=240)
    ap.add_argument("--val", type=int, default=60)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    a = ap.parse_args(argv)
    sys.path.insert(0, ROOT)
    import datagen

    import paper_2404_09276_gb300 as ds

    torch.cuda.init()
    t0 = time.perf_counter()
    recs, Ts, Ws = [], [], []
    Xs = []
    fe = ds.Handle()
    for i in range(a.train):
        rec, T, W, l, k = collect(ds, datagen.TRAIN_SEED0 + i)
        Xs.append(fe.mlp_features(torch.as_tensor(rec, device="cuda"), l, k, P_MAX, TOL).cpu().numpy())
        Ts.append(T)
        Ws.append(W)
    fe.close()
    X, T, W = np.concatenate(Xs), np.concatenate(Ts), np.concatenate(Ws)
    t_collect = time.perf_counter() - t0
    weights, losses = train(ds, X, T, W, steps=a.steps)
    t_train = time.perf_counter() - t0 - t_collect
    val = summarize(compare(ds, [datagen.VAL_SEED0 + i for i in range(a.val)], weights))
    ship = "learned" if val["failures"] == 0 else "plain"
    with open(a.out, "w") as f:
        f.write("# learned shift/stop network of the dashSVD library: 1218 FP32 values\n")
        f.write("# (W1 64 x 16 row-major, b1 64, W2 2 x 64, b2 2)\n")
        f.write(f"# written by: python -m paper_2404_09276_gb300.learn --train {a.train} --val {a.val} "
                f"--steps {a.steps}\n")
        f.write(f"# training: {a.train} matrices (seeds {datagen.TRAIN_SEED0}..), {X.shape[0]} pass records, "
                f"{int((W[:, 1] > 0).sum())} stop decisions ({int(T[W[:, 1] > 0, 1].sum())} positive), "
                f"shift targets {dict(zip(*np.unique(T[:, 0], return_counts=True)))}; collect {t_collect:.0f} s, "
                f"train {t_train:.1f} s; loss {' -> '.join('%.4f' % x for x in losses)}\n")
        f.write(f"# validation: {val['n']} held-out matrices (seeds {datagen.VAL_SEED0}..), tol {TOL}: passes "
                f"plain {val['plain_passes']:.2f} -> learned {val['learned_passes']:.2f}; wall "
                f"plain {val['plain_s']:.3f} s -> learned {val['learned_s']:.3f} s; learned failures "
                f"{val['failures']} {val['fail_seeds']} (runs over tol: plain {val['plain_failures']}, "
                f"both {val['both_over']})\n")
        f.write(f"# ship: {ship}\n")
        for x in weights:
            f.write("%.9g\n" % x)
    print(open(a.out).read().split("\n# ship")[0])
    print("ship:", ship)


if __name__ == "__main__":
    main()
