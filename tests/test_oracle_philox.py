"""Pins for the oracle's Gaussian block (Alg. 5 step 1, Omega = randn(m, l)).

Philox is pinned by the published known-answer vectors; Box-Muller by its
closed forms at special inputs and by distribution tests; the block layout by
slicing identities.
"""
import os

import numpy as np
import pytest
from scipy import stats

from oracle.philox import box_muller, gaussian_block, philox4x32_10

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(w, 16) for w in line.split()])
    return rows


def test_philox_known_answers():
    rows = _kat_rows()
    assert len(rows) == 3
    for r in rows:
        out = philox4x32_10(*r[:4], *r[4:6])
        assert [int(x) for x in out] == r[6:]


def test_philox_vectorised_matches_scalar():
    rng = np.random.default_rng(5)
    w = rng.integers(0, 2**32, size=(6, 17), dtype=np.uint64)
    vec = philox4x32_10(*w)
    for t in range(17):
        one = philox4x32_10(*(int(w[i, t]) for i in range(6)))
        assert [int(vec[i][t]) for i in range(4)] == [int(x) for x in one]


def test_box_muller_closed_forms():
    # w >> 8 == 2^24 - 1 gives u1 = 1 -> radius 0 -> both outputs exactly 0
    z0, z1 = box_muller(0xFFFFFFFF, 12345)
    assert z0 == 0.0 and abs(z1) == 0.0
    # u2 = 0 -> angle 0: (r, 0) with r = sqrt(-2 ln u1)
    wa = (1 << 31)  # (w >> 8) + 1 = 2^23 + 1
    u1 = ((wa >> 8) + 1) * 2.0**-24
    z0, z1 = box_muller(wa, 0)
    assert z0 == pytest.approx(np.sqrt(-2 * np.log(u1)), rel=1e-15) and z1 == 0.0
    # u2 = 1/4 -> angle pi/2: (~0, r)
    z0, z1 = box_muller(wa, 1 << 30)
    assert abs(z0) < 1e-15 and z1 == pytest.approx(np.sqrt(-2 * np.log(u1)), rel=1e-15)


def test_gaussian_block_distribution():
    z = gaussian_block(0x5EED, 50_000, 8)
    flat = z.ravel()
    n = flat.size
    assert abs(flat.mean()) < 5 / np.sqrt(n)
    assert abs(flat.var() - 1) < 5 * np.sqrt(2 / n)
    assert stats.kstest(flat, "norm").pvalue > 1e-3
    c = np.corrcoef(z.T)
    assert np.max(np.abs(c - np.eye(8))) < 5 / np.sqrt(z.shape[0])
    # each of the four output slots of a Philox block is N(0, 1) on its own
    for slot in range(4):
        assert stats.kstest(z[:, slot], "norm").pvalue > 1e-4


def test_gaussian_block_layout():
    full = gaussian_block(7, 40, 10)
    assert full.shape == (40, 10)
    np.testing.assert_array_equal(gaussian_block(7, 15, 10, row0=20), full[20:35])
    np.testing.assert_array_equal(gaussian_block(7, 40, 7), full[:, :7])
    assert not np.allclose(gaussian_block(8, 40, 10), full)
    # entry (i, j) depends only on (seed, i, j >> 2): a 64-bit row index uses the
    # second counter word
    hi = gaussian_block(7, 1, 4, row0=(1 << 32) + 3)
    lo = gaussian_block(7, 1, 4, row0=3)
    assert not np.allclose(hi, lo)
