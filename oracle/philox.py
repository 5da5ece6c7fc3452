"""Philox-4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw 2011,
"Parallel random numbers: as easy as 1, 2, 3", SC'11), written from its
published definition: 10 rounds of two 32x32->64 multiplications by
0xD2511F53 and 0xCD9E8D57 with the key bumped by the Weyl constants
0x9E3779B9 and 0xBB67AE85 between rounds.
"""
from __future__ import annotations

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def philox4x32_10(counter, key):
    """Return the 4 output words for a 4-word counter and a 2-word key."""
    c0, c1, c2, c3 = (int(x) & MASK for x in counter)
    k0, k1 = (int(x) & MASK for x in key)
    for r in range(10):
        if r:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK
        hi1, lo1 = p1 >> 32, p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK, lo1, (hi0 ^ c3 ^ k1) & MASK, lo0
    return c0, c1, c2, c3


def uniform01_from_u32(x):
    """(x >> 8) * 2^-24: a float32-exact uniform on [0, 1)."""
    return (int(x) >> 8) * (1.0 / 16777216.0)
