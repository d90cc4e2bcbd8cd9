"""Sketches SA of the data matrix A (n x d).

SRHT (App. C.2 "Preliminaries" and the proof of Thm 3.2): S = sqrt(n_pad/m) R H_norm
diag(eps), with A zero-padded to n_pad = 2^ceil(log2 n) rows.  The sqrt(n_pad/m)
rescaling is the one the proof of Thm 3.2 applies (v_j = sqrt(n/m) w_j); with it
E[S^T S] = I, which Def 3.2's bounds assume.  Row j of the result is

    SA[j] = (1/sqrt(m)) * sum_{i<n} (-1)^popcount(r_j & i) eps_i a_i ,

r_j the j-th selected row (ascending).

Gaussian (Sec. 1, App. C.1): S has i.i.d. N(0, 1/m) entries and SA = S A.
"""
import numpy as np

from . import rng
from .hadamard import fwht, hadamard_entries, next_pow2


def srht_rows_explicit(A, m, seed, level, which=None):
    """Rows `which` (default all) of the SRHT sketch, each computed as an
    explicit +-1-weighted sum over the n rows of A.  Cost O(len(which) n d);
    suited to sampled checks at any n."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    n_pad = next_pow2(n)
    eps = rng.signs(n_pad, seed, level)[:n].astype(np.float64)
    rows = rng.select_rows(n_pad, m, seed, level)
    if which is None:
        which = np.arange(m)
    which = np.asarray(which)
    out = np.empty((len(which), A.shape[1]), dtype=np.float64)
    for k, j in enumerate(which):
        h = hadamard_entries([rows[j]], np.arange(n))[0]
        out[k] = (h * eps) @ A
    return out / np.sqrt(m)


def srht_sketch(A, m, seed, level):
    """Full SRHT sketch via the plain FWHT of the sign-flipped, zero-padded A."""
    A = np.asarray(A, dtype=np.float64)
    n, d = A.shape
    n_pad = next_pow2(n)
    eps = rng.signs(n_pad, seed, level).astype(np.float64)
    padded = np.zeros((n_pad, d), dtype=np.float64)
    padded[:n] = A
    transformed = fwht(eps[:, None] * padded)
    rows = rng.select_rows(n_pad, m, seed, level)
    return transformed[rows] / np.sqrt(m)


def srht_matrix(n, m, seed, level):
    """Dense S (m x n) of the SRHT, for small n: sqrt(n_pad/m) R H_norm diag(eps)
    restricted to the first n columns."""
    n_pad = next_pow2(n)
    eps = rng.signs(n_pad, seed, level).astype(np.float64)
    rows = rng.select_rows(n_pad, m, seed, level)
    h = hadamard_entries(rows, np.arange(n))
    return h * eps[None, :n] / np.sqrt(m)


def gaussian_sketch(A, m, seed, level, block=8192):
    """SA = S A with S the dense N(0, 1/m) embedding, formed block by block over
    the rows of A (the definition; blocking only bounds memory)."""
    A = np.asarray(A, dtype=np.float64)
    n, d = A.shape
    out = np.zeros((m, d), dtype=np.float64)
    # columns of S (indexed by i < n) are generated independently per counter i
    for i0 in range(0, n, block):
        i1 = min(n, i0 + block)
        z = rng.gaussian_z_cols(m, i0, i1, seed, level)
        out += z @ A[i0:i1]
    return out / np.sqrt(m)


def gaussian_sketch_bf16(A, m, seed, level, block=8192):
    """SA with both operands rounded to BF16 first: (1/sqrt(m)) bf16(z) bf16(A),
    products and sums in float64."""
    from .quant import bf16_round

    A = np.asarray(A, dtype=np.float32)
    n, d = A.shape
    Aq = bf16_round(A).astype(np.float64)
    out = np.zeros((m, d), dtype=np.float64)
    for i0 in range(0, n, block):
        i1 = min(n, i0 + block)
        z = bf16_round(rng.gaussian_z_cols(m, i0, i1, seed, level).astype(np.float32)).astype(np.float64)
        out += z @ Aq[i0:i1]
    return out / np.sqrt(m)


def fp8_column_scales(A):
    """Per-column scales of the E4M3 sketch: s_j = fl32(amax_j / 448) (1 for a
    zero column) and r_j = fl32(1 / s_j), in binary32 as the tensor-core path
    defines them."""
    A = np.asarray(A, dtype=np.float32)
    amax = np.abs(A).max(axis=0).astype(np.float32)
    s = np.where(amax > 0, amax / np.float32(448.0), np.float32(1.0)).astype(np.float32)
    r = (np.float32(1.0) / s).astype(np.float32)
    return s, r


def gaussian_sketch_fp8(A, m, seed, level, block=8192):
    """SA with E4M3 operands and per-column scales:
    (1/sqrt(m)) e4m3(z) e4m3(fl32(A r)) diag(s), sums in float64."""
    from .quant import e4m3_round

    A = np.asarray(A, dtype=np.float32)
    n, d = A.shape
    s, r = fp8_column_scales(A)
    Aq = e4m3_round((A * r[None, :]).astype(np.float32).astype(np.float64))
    out = np.zeros((m, d), dtype=np.float64)
    for i0 in range(0, n, block):
        i1 = min(n, i0 + block)
        z = e4m3_round(rng.gaussian_z_cols(m, i0, i1, seed, level).astype(np.float32).astype(np.float64))
        out += z @ Aq[i0:i1]
    return out * s[None, :].astype(np.float64) / np.sqrt(m)


def sketch(A, m, kind, seed, level):
    if kind == "srht":
        return srht_sketch(A, m, seed, level)
    if kind == "gauss":
        return gaussian_sketch(A, m, seed, level)
    raise ValueError(kind)
