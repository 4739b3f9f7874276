"""ORACLE (test infrastructure): Philox4x32-10 counter-based generator.

Written from its published definition (J. K. Salmon, M. A. Moraes,
R. O. Dror, D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11): a 4x32-bit counter and a 2x32-bit key; each of the 10 rounds does two
32x32->64 multiplications by the round multipliers, mixes the high halves with
the other counter words and the key, and the key is bumped by the Weyl
constants between rounds.  Vectorised over counters with numpy uint64.

The paper itself only states that Clifford fragments are sampled (its sole
error source is sampling error, Sec. V-C); this counter-based generator is how
shots are drawn reproducibly, keyed as described in ``shot_words`` and
``shot_coeffs``.
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


def fields_per_word(rank):
    """Shots one 32-bit output word serves: four 8-bit fields at rank <= 8,
    two 16-bit fields at rank <= 16, else one (rank <= 24)."""
    return 4 if rank <= 8 else 2 if rank <= 16 else 1


def shot_coeffs(n_shots, rank, variant, fragment, circuit, seed_lo, seed_hi):
    """Coefficient bits of each shot of a space of the given rank: shot t takes
    field t mod s (s = fields_per_word(rank), fields from the low bits up, 32/s
    bits each) of word t div s of the ``shot_words`` stream, and uses its low
    rank bits."""
    s = fields_per_word(rank)
    width = 32 // s
    words = shot_words((n_shots + s - 1) // s, variant, fragment, circuit, seed_lo, seed_hi)
    t = np.arange(n_shots, dtype=np.uint64)
    w = words[(t // np.uint64(s)).astype(np.int64)]
    f = (w >> (np.uint64(width) * (t % np.uint64(s)))) & np.uint64((1 << width) - 1)
    return f & np.uint64((1 << rank) - 1)
