"""The seeded input recipes (no method arithmetic): well-formed CSR, the
stated degree and value laws, and determinism by seed, at reduced scale."""
import numpy as np
import pytest

import datagen


def _well_formed(A):
    rp, ci = A.rowptr.astype(np.int64), A.colidx.astype(np.int64)
    assert rp[0] == 0 and rp[-1] == A.nnz == ci.size == A.val.size
    assert np.all(np.diff(rp) >= 0)
    assert ci.min() >= 0 and ci.max() < A.n
    row = np.repeat(np.arange(A.m), np.diff(rp))
    key = row * A.n + ci
    assert np.all(np.diff(key) > 0)  # sorted and unique within each row
    assert A.rowptr.dtype == np.int32 and A.colidx.dtype == np.int32 and A.val.dtype == np.float32


@pytest.mark.parametrize("cfg,scale", [(1, 0.1), (2, 0.002), (3, 0.002), (5, 0.001)])
def test_configs_are_well_formed_and_deterministic(cfg, scale):
    A, prm = datagen.make_config(cfg, scale)
    _well_formed(A)
    B, _ = datagen.make_config(cfg, scale)
    assert np.array_equal(A.colidx, B.colidx) and np.array_equal(A.val, B.val)
    assert prm["k"] >= 1 and prm["s"] >= 1


def test_scaled_gaussian_recipe():
    A, _ = datagen.make_config(1, 0.1)
    deg = np.diff(A.rowptr)
    assert np.all(deg == 20)
    row = np.repeat(np.arange(A.m), deg)
    g = A.val.astype(np.float64) * np.sqrt((row + 1.0) * (A.colidx + 1.0))  # back to the N(0, 1) draws
    assert abs(g.mean()) < 0.02 and abs(g.var() - 1.0) < 0.03


def test_social_graph_recipe():
    A = datagen.social_graph(20_000, 20_000, 7)
    deg = np.diff(A.rowptr)
    assert abs(deg.mean() - 15.0) < 0.1  # bisected mean out-degree
    assert deg.min() >= 1 and deg.max() <= 20_000
    assert np.all(A.val == 1.0)
    indeg = np.bincount(A.colidx, minlength=A.n)
    top = np.sort(indeg)[::-1]
    assert top[:200].sum() > 0.2 * A.nnz  # Zipf(1.1) popularity: a few hot targets
    assert np.argmax(indeg) != 0  # hot columns scattered by the permutation


def test_term_document_and_recommender_values():
    T = datagen.term_document(2000, 5000, 3)
    assert np.all(T.val > 0) and abs(np.log(T.val).std() - 0.75) < 0.02
    R = datagen.recommender(4000, 20_000, 4)
    assert set(np.unique(R.val).tolist()) <= {1.0, 2.0, 3.0, 4.0, 5.0}


def test_powerlaw_degree_bisection():
    rng = np.random.default_rng(1)
    d = datagen._powerlaw_degrees(100_000, 1.2, 50.0, 10_000, rng)
    assert abs(d.mean() - 50.0) < 0.5 and d.max() <= 10_000 and d.min() >= 1


def _distinct_targets_every_round(deg, n, draw, rng, zipf_rounds=12):
    """The redraw loop in its plain form: every round re-sorts all keys."""
    m = deg.size
    deg = np.minimum(deg, n).astype(np.int64)
    keys = np.empty(0, dtype=np.int64)
    need = deg
    rnd = 0
    while True:
        rows = np.repeat(np.arange(m, dtype=np.int64), need)
        if rows.size == 0:
            break
        cols = draw(rows.size, rng) if rnd < zipf_rounds else rng.integers(0, n, rows.size)
        keys = np.unique(np.concatenate([keys, rows * n + cols]))
        need = np.maximum(deg - np.bincount(keys // n, minlength=m), 0)
        rnd += 1
    return keys


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_redraw_rounds_set_complete_rows_aside(seed):
    """The generator's redraw rounds set complete rows aside: the same draws
    and the same keys as the plain loop, including rows that need every
    column (uniform rounds after the Zipf ones)."""
    m, n = 300, 40
    rng0 = np.random.default_rng(seed)
    deg = np.minimum(rng0.integers(0, 60, m), n)
    deg[:5] = n
    zipf = datagen._ZipfSampler(n, 1.2)
    a = datagen._distinct_targets(deg, n, lambda k, g: zipf(k, g), np.random.default_rng(seed + 10))
    b = _distinct_targets_every_round(deg, n, lambda k, g: zipf(k, g), np.random.default_rng(seed + 10))
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(np.bincount(a // n, minlength=m), np.minimum(deg, n))


def test_exact_fill_gives_every_row_its_degree():
    """fill_exact: rows still short after the Zipf rounds take their deficit
    without replacement from the columns they lack (distinct, in range)."""
    m, n = 200, 50
    deg = np.full(m, 10)
    deg[:20] = n
    zipf = datagen._ZipfSampler(n, 1.4)
    keys = datagen._distinct_targets(deg, n, lambda k, g: zipf(k, g), np.random.default_rng(5), fill_exact=True)
    assert np.all(np.diff(keys) > 0)
    np.testing.assert_array_equal(np.bincount(keys // n, minlength=m), deg)
    assert keys.min() >= 0 and keys.max() < m * n
