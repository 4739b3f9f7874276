"""ORACLE (test infrastructure): Philox4x32-10 counter-based generator.

Written from its published definition (J. K. Salmon, M. A. Moraes,
R. O. Dror, D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11): a 4x32-bit counter and a 2x32-bit key; each of the 10 rounds does two
32x32->64 multiplications by the round multipliers, mixes the high halves with
the other counter words and the key, and the key is bumped by the Weyl
constants between rounds.  Vectorised over counters with numpy uint64.

The paper itself only states that Clifford fragments are sampled (its sole
error source is sampling error, Sec. V-C); this counter-based generator is how
shots are drawn reproducibly, keyed as described in ``shot_words``.
"""
from __future__ import annotations

import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57           # round multipliers
W0, W1 = 0x9E3779B9, 0xBB67AE85           # key increments (Weyl sequence)
_MASK = 0xFFFFFFFF


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Return the four 32-bit output words (uint64 arrays holding uint32)."""
    c0 = np.asarray(c0, np.uint64) & _MASK
    c1 = np.asarray(c1, np.uint64) & _MASK
    c2 = np.asarray(c2, np.uint64) & _MASK
    c3 = np.asarray(c3, np.uint64) & _MASK
    k0, k1 = int(k0) & _MASK, int(k1) & _MASK
    for rnd in range(10):
        if rnd:
            k0 = (k0 + W0) & _MASK
            k1 = (k1 + W1) & _MASK
        p0 = np.uint64(M0) * c0
        p1 = np.uint64(M1) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(_MASK)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(_MASK)
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1,
                          hi0 ^ c3 ^ np.uint64(k1), lo0)
    return c0, c1, c2, c3


def shot_words(n_shots, variant, fragment, circuit, seed_lo, seed_hi):
    """32 random bits per shot: key = (seed_lo, seed_hi); shot s takes output
    word s mod 4 of the block with counter (s div 4, variant, fragment,
    circuit), so one generator call serves four consecutive shots."""
    g = np.arange((n_shots + 3) // 4, dtype=np.uint64)
    w = philox4x32_10(g, np.full_like(g, variant), np.full_like(g, fragment),
                      np.full_like(g, circuit), seed_lo, seed_hi)
    return np.stack(w, axis=1).reshape(-1)[:n_shots]
