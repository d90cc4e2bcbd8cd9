"""Philox4x32-10, written from its published definition.

Reference: J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11 (Sec. 4.2, the Philox S-box).  A round maps
the 4x32-bit counter (c0, c1, c2, c3) with key (k0, k1) through two 32x32->64
multiplies:

    (hi0, lo0) = M0 * c0        (hi1, lo1) = M1 * c2
    c' = (hi1 ^ c1 ^ k0,  lo1,  hi0 ^ c3 ^ k1,  lo0)

and the key is advanced by the Weyl constants (W0, W1) between rounds.  Ten
rounds.  Pinned by the known-answer vectors in ``tests/golden``.

The paper itself leaves the random source unspecified; this generator is the
project's reading (random draws must be reproducible on both sides of the
parity tests).
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)
SHIFT = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Apply ten Philox rounds.  Counter words are arrays (broadcast together) of
    values < 2**32; key words are scalars.  Returns four uint64 arrays holding the
    32-bit output words."""
    c0 = np.asarray(c0, dtype=np.uint64) & MASK
    c1 = np.asarray(c1, dtype=np.uint64) & MASK
    c2 = np.asarray(c2, dtype=np.uint64) & MASK
    c3 = np.asarray(c3, dtype=np.uint64) & MASK
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> SHIFT, p0 & MASK
        hi1, lo1 = p1 >> SHIFT, p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return c0, c1, c2, c3


def seed_key(seed):
    """Key words of a 64-bit seed: (low 32 bits, high 32 bits)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32
