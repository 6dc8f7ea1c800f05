"""Seeded synthetic sparse inputs for the dashSVD hot path.

This module only draws matrices: structure (row degrees, column ids) and
values, from numpy's PCG64 generator with a fixed seed. It holds none of the
method's arithmetic and is shared by the FP64 oracle, the GPU tests and the
benchmark, so that both sides of a parity check see the same matrix.

The paper evaluates on real matrices (social graphs, a recommender matrix,
term-document matrices; Sec. 4, Table 1). None of them is available here; the
recipes below stand in for their shapes:

* ``scaled_gaussian``  -- uniform random support, values g*(i+1)^-1/2*(j+1)^-1/2
* ``social_graph``     -- power-law out-degrees, Zipf target popularity, 0/1
* ``term_document``    -- lognormal row lengths, Zipf column ids, lognormal values
* ``recommender``      -- power-law user degrees, Zipf item popularity, {1..5}

All matrices are CSR with int32 row pointers and column ids (sorted and unique
within a row) and float32 values.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = [
    "Csr",
    "scaled_gaussian",
    "social_graph",
    "term_document",
    "training_matrix",
    "recommender",
    "dense_as_csr",
    "dense_with_spectrum",
    "CONFIGS",
    "make_config",
]


@dataclass
class Csr:
    """A CSR matrix held in host memory (int32 indices, float32 values)."""

    m: int
    n: int
    rowptr: np.ndarray  # int32, shape (m + 1,)
    colidx: np.ndarray  # int32, shape (nnz,)
    val: np.ndarray  # float32, shape (nnz,)
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.colidx.size)

    def to_scipy(self, dtype=np.float64):
        import scipy.sparse as sp

        return sp.csr_matrix(
            (self.val.astype(dtype), self.colidx, self.rowptr), shape=(self.m, self.n)
        )

    def to_dense(self, dtype=np.float64) -> np.ndarray:
        return self.to_scipy(dtype).toarray()

    def nbytes(self) -> int:
        return self.rowptr.nbytes + self.colidx.nbytes + self.val.nbytes


def _dedup_sorted(keys: np.ndarray) -> np.ndarray:
    """Sort int64 keys (timsort: fast on concatenated sorted runs) and drop repeats."""
    keys = np.sort(keys, kind="stable")
    if keys.size:
        keep = np.empty(keys.size, dtype=bool)
        keep[0] = True
        np.not_equal(keys[1:], keys[:-1], out=keep[1:])
        keys = keys[keep]
    return keys


def _csr_from_keys(m: int, n: int, keys: np.ndarray, vals_fn, rng, name: str) -> Csr:
    """Build CSR from sorted unique keys row*n + col, then draw the values."""
    r = keys // n
    c = (keys - r * n).astype(np.int32)
    counts = np.bincount(r, minlength=m)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32 row pointers")
    vals = vals_fn(r, c, rng).astype(np.float32)
    return Csr(m, n, rowptr.astype(np.int32), c, vals, name)


class _ZipfSampler:
    """Discrete Zipf ranks 0..n-1, P(r) proportional to (r+1)^-s, by inverse CDF
    with a guide table (Chen and Asau) so that a draw costs O(1) on average."""

    def __init__(self, n: int, s: float):
        w = np.arange(1, n + 1, dtype=np.float64) ** (-s)
        self.cdf = np.cumsum(w)
        self.cdf /= self.cdf[-1]
        self.cdf[-1] = 1.0
        self.nb = 1 << max(10, int(np.ceil(np.log2(n))) + 1)
        self.guide = np.searchsorted(self.cdf, np.arange(self.nb) / self.nb, side="right")

    def __call__(self, count: int, rng) -> np.ndarray:
        u = rng.random(count)
        r = self.guide[np.minimum((u * self.nb).astype(np.int64), self.nb - 1)]
        todo = np.nonzero(self.cdf[r] <= u)[0]
        while todo.size:
            r[todo] += 1
            todo = todo[self.cdf[r[todo]] <= u[todo]]
        return r


def _distinct_targets(deg: np.ndarray, n: int, draw, rng, zipf_rounds: int = 12,
                      fill_exact: bool = False) -> np.ndarray:
    """Give row i exactly min(deg[i], n) distinct targets.

    Targets are drawn with ``draw(count, rng)``. Rows that lost draws to
    duplicates are topped up for ``zipf_rounds`` rounds; any deficit left after
    that (only very long rows, which have used up the popular targets) is
    filled with uniformly drawn targets: by further rounds of draws with
    replacement, or, with ``fill_exact``, in one step, each short row taking
    its deficit as a uniform draw without replacement from the columns it
    lacks (rows that need almost every column would otherwise take a round per
    missing column, as in coupon collecting). Returns sorted keys row*n + col.

    Rows that are complete are set aside after each round, so that the
    top-up rounds (many, for rows that need almost every column) only sort
    the keys of the rows still short; the draws and the result are the same
    as when every round works on all keys.
    """
    m = deg.size
    deg = np.minimum(deg, n).astype(np.int64)
    done = []  # sorted keys of complete rows
    keys = np.empty(0, dtype=np.int64)  # sorted keys of the rows still short
    need = deg
    rnd = 0
    while True:
        rows = np.repeat(np.arange(m, dtype=np.int64), need)
        if rows.size == 0:
            break
        if fill_exact and rnd == zipf_rounds:
            fill = []
            for r in np.nonzero(need)[0]:
                lo, hi = np.searchsorted(keys, [r * n, (r + 1) * n])
                lack = np.setdiff1d(np.arange(n, dtype=np.int64), keys[lo:hi] - r * n, assume_unique=True)
                fill.append(r * n + np.sort(rng.choice(lack, int(need[r]), replace=False)))
            done.append(keys)
            done.extend(fill)
            keys = np.empty(0, dtype=np.int64)
            break
        cols = draw(rows.size, rng) if rnd < zipf_rounds else rng.integers(0, n, rows.size)
        keys = _dedup_sorted(np.concatenate([keys, _dedup_sorted(rows * n + cols)]))
        have = np.bincount(keys // n, minlength=m)
        short = np.zeros(m, dtype=bool)
        short[np.nonzero(need)[0]] = True  # only rows drawn this round can be short or newly complete
        need = np.where(short, np.maximum(deg - have, 0), 0)
        complete = (keys // n)
        sel = short[complete] & (need[complete] == 0)
        if sel.any():
            done.append(keys[sel])
            keys = keys[~sel]
        rnd += 1
    if done:
        keys = _dedup_sorted(np.concatenate(done + [keys]))
    return keys


def _powerlaw_degrees(m: int, tail: float, mean: float, dmax: int, rng) -> np.ndarray:
    """Degrees d = min(dmax, ceil(x_min * U^(-1/tail))), x_min bisected so mean(d) ~= mean.

    ``tail`` is the exponent of the complementary CDF (a density exponent of
    tail + 1). The same uniforms are reused during bisection, so the result is a
    deterministic function of the seed.
    """
    u = 1.0 - rng.random(m)  # (0, 1]
    base = u ** (-1.0 / tail)
    lo, hi = 1e-6, float(mean)
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if np.minimum(dmax, np.ceil(mid * base)).mean() < mean:
            lo = mid
        else:
            hi = mid
    return np.minimum(dmax, np.ceil(hi * base)).astype(np.int64)


def scaled_gaussian(m: int, n: int, per_row: int, seed: int, name: str = "scaled_gaussian") -> Csr:
    """Each row holds ``per_row`` distinct uniformly drawn columns (duplicates are
    redrawn); a_ij = g_ij * (i+1)^-1/2 * (j+1)^-1/2 with g_ij ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    deg = np.full(m, min(per_row, n), dtype=np.int64)
    keys = _distinct_targets(deg, n, lambda k, g: g.integers(0, n, k), rng)

    def vals(r, c, g):
        return g.standard_normal(r.size) * (r + 1.0) ** -0.5 * (c + 1.0) ** -0.5

    return _csr_from_keys(m, n, keys, vals, rng, name)


def social_graph(
    m: int, n: int, seed: int, mean_degree: float = 15.0, degree_tail: float = 1.1,
    max_degree: int = 50_000, popularity: float = 1.1, name: str = "social_graph",
) -> Csr:
    """Binary adjacency: power-law out-degrees (CCDF exponent ``degree_tail``,
    i.e. density exponent 2.1 by default), distinct targets drawn with Zipf
    popularity through a seeded permutation (hot columns scattered)."""
    rng = np.random.default_rng(seed)
    deg = _powerlaw_degrees(m, degree_tail, mean_degree, min(max_degree, n), rng)
    perm = rng.permutation(n)
    zipf = _ZipfSampler(n, popularity)
    keys = _distinct_targets(deg, n, lambda k, g: perm[zipf(k, g)], rng)
    return _csr_from_keys(m, n, keys, lambda r, c, g: np.ones(r.size), rng, name)


def term_document(
    m: int, n: int, seed: int, mean_len: float = 100.0, sigma: float = 1.0,
    popularity: float = 1.1, value_sigma: float = 0.75, name: str = "term_document",
) -> Csr:
    """Row lengths round(LogNormal(ln(mean) - sigma^2/2, sigma)) clamped to [1, n];
    distinct Zipf column ids through a permutation; values LogNormal(0, value_sigma)."""
    rng = np.random.default_rng(seed)
    mu = np.log(mean_len) - 0.5 * sigma * sigma
    lens = np.clip(np.rint(rng.lognormal(mu, sigma, m)), 1, n).astype(np.int64)
    perm = rng.permutation(n)
    zipf = _ZipfSampler(n, popularity)
    keys = _distinct_targets(lens, n, lambda k, g: perm[zipf(k, g)], rng)
    return _csr_from_keys(
        m, n, keys, lambda r, c, g: g.lognormal(0.0, value_sigma, r.size), rng, name
    )


def recommender(
    m: int, n: int, seed: int, mean_degree: float = 50.0, degree_tail: float = 1.2,
    popularity: float = 1.2, name: str = "recommender", max_degree: int | None = None,
    fill_exact: bool = False,
) -> Csr:
    """User-item ratings: power-law user degrees (capped at ``max_degree``, default
    n), distinct Zipf items through a permutation, ratings uniform in {1, ..., 5}.
    ``fill_exact``: see _distinct_targets (the benchmark workload, whose
    longest rows need almost every column, uses it)."""
    rng = np.random.default_rng(seed)
    deg = _powerlaw_degrees(m, degree_tail, mean_degree, n if max_degree is None else min(max_degree, n), rng)
    perm = rng.permutation(n)
    zipf = _ZipfSampler(n, popularity)
    keys = _distinct_targets(deg, n, lambda k, g: perm[zipf(k, g)], rng, fill_exact=fill_exact)
    return _csr_from_keys(
        m, n, keys, lambda r, c, g: g.integers(1, 6, r.size).astype(np.float64), rng, name
    )


def dense_as_csr(a: np.ndarray, name: str = "dense") -> Csr:
    """Store a dense array in CSR (explicit zeros dropped)."""
    a = np.asarray(a)
    m, n = a.shape
    r, c = np.nonzero(a)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=m), out=rowptr[1:])
    return Csr(m, n, rowptr.astype(np.int32), c.astype(np.int32), a[r, c].astype(np.float32), name)


def dense_with_spectrum(m: int, n: int, sigma: np.ndarray, seed: int) -> np.ndarray:
    """Dense m x n matrix U diag(sigma) V^T with Haar-like random orthonormal U, V
    (QR of Gaussian blocks). ``sigma`` has min(m, n) entries. This builds the
    paper's "Dense2" test case (sigma_i = 1/sqrt(i), Sec. 4) and other inputs with
    a known spectrum."""
    rng = np.random.default_rng(seed)
    r = min(m, n)
    U, _ = np.linalg.qr(rng.standard_normal((m, r)))
    V, _ = np.linalg.qr(rng.standard_normal((n, r)))
    return (U * np.asarray(sigma, dtype=np.float64)[None, :]) @ V.T


# The five workloads: matrix recipe, seed 1000 + config number, and the
# run parameters (k, s, max passes, PVE tolerance).
CONFIGS = {
    1: dict(kind="scaled_gaussian", m=20_000, n=10_000, per_row=20, k=20, s=10, p_max=10, tol=1e-2),
    2: dict(kind="social_graph", m=1_000_000, n=1_000_000, k=100, s=50, p_max=20, tol=1e-2),
    3: dict(kind="term_document", m=500_000, n=100_000, k=100, s=50, p_max=20, tol=1e-2),
    4: dict(kind="term_document", m=500_000, n=100_000, k=100, s=50, p_max=20, tol=1e-2),
    5: dict(kind="recommender", m=2_000_000, n=200_000, k=200, s=20, p_max=20, tol=1e-2),
}


# Training and validation family of the learned form: seeds 10,000.. are the
# training matrices and 20,000.. the held-out ones (disjoint by construction).
TRAIN_SEED0, VAL_SEED0 = 10_000, 20_000


def training_matrix(seed: int, m_range=(10_000, 60_000)) -> tuple[Csr, dict]:
    """One member of the learned form's matrix family: a power-law social graph,
    a recommender or a term-document matrix (chosen by the seed), with m drawn
    uniformly from ``m_range``, n = m * U[1/4, 1], the degree mean, tails and
    popularity drawn per matrix, and k in {20, 50, 100} with s = k / 2."""
    rng = np.random.default_rng(seed)
    m = int(rng.integers(m_range[0], m_range[1] + 1))
    n = max(400, int(m * rng.uniform(0.25, 1.0)))
    kind = ("social_graph", "recommender", "term_document")[int(rng.integers(0, 3))]
    k = int((20, 50, 100)[int(rng.integers(0, 3))])
    sub = int(rng.integers(0, 2**31))
    if kind == "social_graph":
        A = social_graph(m, n, sub, mean_degree=float(rng.uniform(8, 25)), degree_tail=float(rng.uniform(1.05, 1.5)),
                         max_degree=n // 8, popularity=float(rng.uniform(0.9, 1.3)), name="train_social")
    elif kind == "recommender":
        A = recommender(m, n, sub, mean_degree=float(rng.uniform(15, 50)), degree_tail=float(rng.uniform(1.1, 1.6)),
                        popularity=float(rng.uniform(0.9, 1.4)), name="train_recommender", max_degree=n // 8)
    else:
        A = term_document(m, n, sub, mean_len=float(rng.uniform(20, 60)), sigma=float(rng.uniform(0.6, 1.2)),
                          popularity=float(rng.uniform(0.9, 1.3)), name="train_term_document")
    return A, dict(kind=kind, k=k, s=k // 2, p_max=20, tol=1e-2)


def make_config(cfg: int, scale: float = 1.0) -> tuple[Csr, dict]:
    """Build the matrix of workload ``cfg`` (seed 1000 + cfg).

    ``scale`` < 1 shrinks m and n by that factor with the same recipe, for
    cases the oracle finishes in seconds. Returns (matrix, run parameters).
    """
    c = dict(CONFIGS[cfg])
    kind = c.pop("kind")
    m = max(1, int(round(c.pop("m") * scale)))
    n = max(1, int(round(c.pop("n") * scale)))
    seed = 1000 + cfg
    tag = f"cfg{cfg}" + ("" if scale == 1.0 else f"x{scale:g}")
    if kind == "scaled_gaussian":
        A = scaled_gaussian(m, n, c.pop("per_row"), seed, name=tag)
    elif kind == "social_graph":
        A = social_graph(m, n, seed, max_degree=max(1, min(50_000, n)), name=tag)
    elif kind == "term_document":
        A = term_document(m, n, seed, name=tag)
    else:
        A = recommender(m, n, seed, name=tag, fill_exact=True)
    return A, c
