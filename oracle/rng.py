"""Seeded random draws of the method, as a specification both sides implement.

The paper needs three random objects and fixes their distributions but not their
source:

* Rademacher signs eps_i, i < n_pad (SRHT, App. C.2 "Preliminaries":
  S = R H diag(eps));
* a subset of m row indices of [0, n_pad) drawn uniformly without replacement
  (App. C.2, matrix Bernstein without replacement);
* i.i.d. N(0, 1/m) entries of a Gaussian embedding (Sec. 1; App. C.1).

Counter layout (Philox4x32-10, key = (seed_lo, seed_hi)):

    stream SIGNS = 0 : rows are grouped in blocks of 1024; block b owns the 32
                       words of Philox counters 8b .. 8b+7 (counter (c_lo, c_hi,
                       level, 0); word 4t + k is output word k of counter 8b + t).
                       Row i = 1024 b + q takes bit (q >> 5) of word (q & 31):
                       eps_i = +1 if that bit is 0 else -1
    stream ROWS  = 1 : counter (i_lo, i_hi, level, 1)     -> key_i = (w1 << 32) | w0
    stream GAUSS = 2 : counter (i, q, level, 2), q = j//4 -> z[4q .. 4q+3, i] by Box-Muller

Row subset: the m indices i with the smallest (key_i, i) pairs (lexicographic),
returned in ascending index order.  With independent uniform 64-bit keys this is
a uniformly random m-subset.  The order of SA's rows is immaterial to H_S
(A^T S^T S A is invariant under row permutations of S); ascending index order is
this project's choice so that parity is element by element.

Gaussian entries: with u1 = (floor(w/2^8) + 1) 2^-24 in (0, 1] and
u2 = floor(w'/2^8) 2^-24 in [0, 1) (both exact in binary32 and binary64),
z = sqrt(-2 ln u1) cos(2 pi u2) and z' = sqrt(-2 ln u1) sin(2 pi u2)
(Box & Muller 1958).  Words (w0, w1) give rows 4q and 4q+1, (w2, w3) give rows
4q+2 and 4q+3.  The sketch entry is S[j, i] = z[j, i] / sqrt(m).
"""
import numpy as np

from .philox import philox4x32_10, seed_key

SIGNS, ROWS, GAUSS = 0, 1, 2


def _split_index(i):
    i = np.asarray(i, dtype=np.uint64)
    return i & np.uint64(0xFFFFFFFF), i >> np.uint64(32)


def signs(n_pad, seed, level):
    """Rademacher vector eps in {-1, +1}^n_pad (int8): row i = 1024 b + q takes
    bit (q >> 5) of word (q & 31) of block b's 32 Philox words."""
    k0, k1 = seed_key(seed)
    blocks = (n_pad + 1023) // 1024
    ctr = np.arange(8 * blocks, dtype=np.uint64)
    lo, hi = _split_index(ctr)
    w = philox4x32_10(lo, hi, np.uint64(level), np.uint64(SIGNS), k0, k1)
    words = np.stack(w, axis=1).reshape(blocks, 32)   # word 4t + k of block b
    i = np.arange(n_pad, dtype=np.int64)
    q = i % 1024
    word = words[i // 1024, q % 32]
    bit = (word >> (q // 32).astype(np.uint64)) & np.uint64(1)
    return (1 - 2 * bit.astype(np.int64)).astype(np.int8)


def row_keys(n_pad, seed, level):
    """64-bit selection keys of every candidate row 0..n_pad-1 (uint64)."""
    k0, k1 = seed_key(seed)
    lo, hi = _split_index(np.arange(n_pad, dtype=np.uint64))
    w0, w1, _, _ = philox4x32_10(lo, hi, np.uint64(level), np.uint64(ROWS), k0, k1)
    return (w1 << np.uint64(32)) | w0


def select_rows(n_pad, m, seed, level):
    """The m row indices of [0, n_pad) with the smallest (key, index) pairs,
    in ascending index order (int64)."""
    if not 1 <= m <= n_pad:
        raise ValueError("need 1 <= m <= n_pad")
    keys = row_keys(n_pad, seed, level)
    order = np.lexsort((np.arange(n_pad), keys))  # primary key: keys, then index
    return np.sort(order[:m]).astype(np.int64)


def _uniform_open0(w):
    """(floor(w / 2^8) + 1) * 2^-24, in (0, 1]."""
    return ((w >> np.uint64(8)).astype(np.float64) + 1.0) * 2.0 ** -24


def _uniform_closed0(w):
    """floor(w / 2^8) * 2^-24, in [0, 1)."""
    return (w >> np.uint64(8)).astype(np.float64) * 2.0 ** -24


def gaussian_z_cols(m, i0, i1, seed, level):
    """Standard normal draws z[j, i] for j < m and columns i0 <= i < i1
    (float64, m x (i1 - i0)); the Gaussian embedding is S = z / sqrt(m)."""
    k0, k1 = seed_key(seed)
    q_count = (m + 3) // 4
    i = np.arange(i0, i1, dtype=np.uint64)[None, :]
    q = np.arange(q_count, dtype=np.uint64)[:, None]
    w0, w1, w2, w3 = philox4x32_10(i, q, np.uint64(level), np.uint64(GAUSS), k0, k1)
    z = np.empty((4 * q_count, i1 - i0), dtype=np.float64)
    for (wa, wb), r0 in (((w0, w1), 0), ((w2, w3), 2)):
        radius = np.sqrt(-2.0 * np.log(_uniform_open0(wa)))
        angle = 2.0 * np.pi * _uniform_closed0(wb)
        z[r0::4] = radius * np.cos(angle)
        z[r0 + 1::4] = radius * np.sin(angle)
    return z[:m]


def gaussian_z_rows(rows, n, seed, level):
    """Selected rows j of the standard normal draws, all n columns
    (len(rows) x n); for sampled checks at large n."""
    k0, k1 = seed_key(seed)
    out = np.empty((len(rows), n), dtype=np.float64)
    i = np.arange(n, dtype=np.uint64)
    for k, j in enumerate(rows):
        w = philox4x32_10(i, np.uint64(j // 4), np.uint64(level), np.uint64(GAUSS), k0, k1)
        lane = j % 4
        wa, wb = (w[0], w[1]) if lane < 2 else (w[2], w[3])
        radius = np.sqrt(-2.0 * np.log(_uniform_open0(wa)))
        angle = 2.0 * np.pi * _uniform_closed0(wb)
        out[k] = radius * (np.cos(angle) if lane % 2 == 0 else np.sin(angle))
    return out


def gaussian_z(m, n, seed, level):
    """All n columns of the standard normal draws (m x n)."""
    return gaussian_z_cols(m, 0, n, seed, level)


def gaussian_embedding(m, n, seed, level):
    """Dense S in R^{m x n}, i.i.d. N(0, 1/m) (Sec. 1)."""
    return gaussian_z(m, n, seed, level) / np.sqrt(m)
