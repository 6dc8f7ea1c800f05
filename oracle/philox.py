"""Counter-based Gaussian block for the oracle (FP64).

TEST INFRASTRUCTURE: this file belongs to the oracle, which only the tests,
the benchmark's CPU-baseline leg and the smoke check may use.

dashSVD draws a Gaussian i.i.d. block Omega (Alg. 5, step 1: Omega = randn(m, l)).
Any i.i.d. N(0, 1) source is a valid reading of "randn"; both sides of the
parity check use the same counter-based generator so that they see the same
Omega without storing it:

* Philox4x32-10, the counter-based generator of Salmon, Moraes, Dror and
  Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of
  two 32x32->64-bit multiplications on a 128-bit counter with a 64-bit key
  that is bumped by the Weyl constants between rounds.
* Box-Muller (1958) turns two uniforms into two independent normals.

Layout of Omega (m x l): entry (i, j) comes from the Philox block with
counter (i mod 2^32, i >> 32, j >> 2, 0) and key (seed mod 2^32, seed >> 32).
Output words (w0, w1) feed columns 4q and 4q+1 (cosine, sine branch) and
(w2, w3) feed 4q+2 and 4q+3. The uniforms are u1 = ((w >> 8) + 1) * 2^-24 in
(0, 1] (radius) and u2 = (w >> 8) * 2^-24 in [0, 1) (angle); both are exact
in FP32 and FP64, so the two sides differ only in the rounding of
sqrt(-2 ln u1) * cos/sin(2 pi u2).
"""
from __future__ import annotations

import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on uint32 arrays (broadcastable).

    Each round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2 as 64-bit products;
    the new counter is (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0). The key is
    bumped by (W0, W1) after every round but the last.
    """
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & _MASK for x in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    m0 = np.uint64(PHILOX_M0)
    m1 = np.uint64(PHILOX_M1)
    for r in range(10):
        p0 = c0 * m0
        p1 = c2 * m1
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        if r < 9:
            k0 = (k0 + np.uint64(PHILOX_W0)) & _MASK
            k1 = (k1 + np.uint64(PHILOX_W1)) & _MASK
    return tuple(x.astype(np.uint32) for x in (c0, c1, c2, c3))


def box_muller(wa, wb):
    """Two independent N(0, 1) values from two uint32 words (FP64)."""
    wa = np.asarray(wa, dtype=np.uint32)
    wb = np.asarray(wb, dtype=np.uint32)
    u1 = ((wa >> np.uint32(8)).astype(np.float64) + 1.0) * 2.0**-24
    u2 = (wb >> np.uint32(8)).astype(np.float64) * 2.0**-24
    r = np.sqrt(-2.0 * np.log(u1))
    t = 2.0 * np.pi * u2
    return r * np.cos(t), r * np.sin(t)


def gaussian_block(seed: int, rows: int, cols: int, row0: int = 0) -> np.ndarray:
    """Rows row0 .. row0+rows-1 of Omega with ``cols`` columns (FP64)."""
    q = (cols + 3) // 4
    i = np.arange(row0, row0 + rows, dtype=np.uint64)[:, None]
    jq = np.arange(q, dtype=np.uint64)[None, :]
    w0, w1, w2, w3 = philox4x32_10(
        i & _MASK, i >> np.uint64(32), jq, np.zeros_like(jq),
        np.uint64(seed) & _MASK, np.uint64(seed) >> np.uint64(32),
    )
    z0, z1 = box_muller(w0, w1)
    z2, z3 = box_muller(w2, w3)
    out = np.empty((rows, 4 * q), dtype=np.float64)
    out[:, 0::4] = z0
    out[:, 1::4] = z1
    out[:, 2::4] = z2
    out[:, 3::4] = z3
    return out[:, :cols]
