"""Walsh-Hadamard transform used by the SRHT (App. C.2, "Preliminaries").

Natural (Sylvester) ordering: the unnormalised matrix has entries
H[r, i] = (-1)^popcount(r & i); the normalised transform of App. C.2 is
H / sqrt(n_pad), which satisfies H_norm^2 = I (used in the proof of Thm 3.2).
The paper does not fix an ordering; any other ordering permutes rows, which the
uniform row subsample makes immaterial.
"""
import numpy as np


def next_pow2(n):
    p = 1
    while p < n:
        p *= 2
    return p


def popcount(v):
    v = np.asarray(v, dtype=np.uint64)
    count = np.zeros(v.shape, dtype=np.int64)
    while np.any(v):
        count += (v & np.uint64(1)).astype(np.int64)
        v = v >> np.uint64(1)
    return count


def hadamard_entries(rows, cols):
    """Unnormalised entries (-1)^popcount(r & i) for the outer grid rows x cols."""
    r = np.asarray(rows, dtype=np.uint64)[:, None]
    i = np.asarray(cols, dtype=np.uint64)[None, :]
    return (1 - 2 * (popcount(r & i) & 1)).astype(np.float64)


def hadamard(n_pad):
    """Explicit unnormalised n_pad x n_pad Hadamard matrix (small n_pad only)."""
    idx = np.arange(n_pad)
    return hadamard_entries(idx, idx)


def fwht(x):
    """Unnormalised fast Walsh-Hadamard transform along axis 0 (length a power of
    two): returns H @ x by log2(n) butterfly stages (a+b, a-b)."""
    y = np.array(x, dtype=np.float64, copy=True)
    n = y.shape[0]
    if n & (n - 1):
        raise ValueError("length must be a power of two")
    h = 1
    while h < n:
        y = y.reshape((n // (2 * h), 2, h) + y.shape[1:])
        a = y[:, 0].copy()
        b = y[:, 1]
        y[:, 0] = a + b
        y[:, 1] = a - b
        y = y.reshape((n,) + y.shape[3:])
        h *= 2
    return y
