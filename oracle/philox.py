"""Counter-based Gaussian random numbers for the sampling matrix R.

The paper fills R element by element from a generator re-seeded per global
row index, so that siblings and parents agree on shared rows (Section
2.2.2 and Section 4.3, eq. Rmerge and the extend-merge figure).  Reading
taken here: a counter-based generator keyed by the seed and addressed by
(global row, column) gives the same property with no state at all:

    G(seed, g, c) = sqrt(-2 ln u1) * cos(2 pi u2),
    (x0, x1, _, _) = Philox4x32-10(key = (seed_lo, seed_hi), ctr = (g, c, 0, 0)),
    u_i = (x_i + 0.5) * 2^-32.

Philox4x32-10 is the generator of Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC'11), written here from
that definition: ten rounds, each multiplying two counter words by the
round multipliers, xoring the high halves with the other two words and the
key, and bumping the key by the Weyl constants between rounds.
"""
from __future__ import annotations

import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds.

    ctr: uint array of shape (..., 4) (values < 2^32), key: (..., 2).
    Returns uint64 array of shape (..., 4) holding 32-bit words.
    """
    c = np.asarray(ctr, dtype=np.uint64) & _MASK
    k = np.asarray(key, dtype=np.uint64) & _MASK
    c0, c1, c2, c3 = (c[..., i].copy() for i in range(4))
    k0 = np.broadcast_to(k[..., 0], c0.shape).copy()
    k1 = np.broadcast_to(k[..., 1], c0.shape).copy()
    m0 = np.uint64(PHILOX_M0)
    m1 = np.uint64(PHILOX_M1)
    for r in range(10):
        if r > 0:
            k0 = (k0 + np.uint64(PHILOX_W0)) & _MASK
            k1 = (k1 + np.uint64(PHILOX_W1)) & _MASK
        p0 = c0 * m0  # exact: both factors < 2^32
        p1 = c2 * m1
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1)


def gaussian(seed, rows, cols):
    """R entries G(seed, g, c) for global rows ``rows`` and columns ``cols``.

    Returns a float64 array of shape (len(rows), len(cols)).
    """
    rows = np.asarray(rows, dtype=np.uint64).reshape(-1)
    cols = np.asarray(cols, dtype=np.uint64).reshape(-1)
    g, c = np.meshgrid(rows, cols, indexing="ij")
    ctr = np.stack([g, c, np.zeros_like(g), np.zeros_like(g)], axis=-1)
    seed = int(seed)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)
    out = philox4x32_10(ctr, key)
    u1 = (out[..., 0].astype(np.float64) + 0.5) * 2.0 ** -32
    u2 = (out[..., 1].astype(np.float64) + 0.5) * 2.0 ** -32
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
