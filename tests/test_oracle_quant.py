"""Pins of the low-precision rounding used by the tensor-core sketch: against
torch's CPU conversions (library routines) and by construction."""
import numpy as np
import pytest

from oracle import quant

torch = pytest.importorskip("torch")


def test_bf16_matches_torch():
    x = np.random.default_rng(0).standard_normal(100000).astype(np.float32) * 10 ** np.random.default_rng(1).uniform(-5, 5, 100000).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(quant.bf16_round(x), ref)


def test_bf16_ties_to_even():
    # 1 + 2^-8 is halfway between bf16 neighbours 1 and 1 + 2^-7: rounds to the even one (1)
    x = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8], dtype=np.float32)
    assert list(quant.bf16_round(x)) == [1.0, 1 + 2 * 2.0 ** -7]


def test_e4m3_table_and_torch():
    vals = quant._E4M3
    assert vals[-1] == 448.0 and vals[0] == 0.0 and len(vals) == 127   # 126 positive finite codes + zero
    x = np.random.default_rng(2).uniform(-440, 440, 50000)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(quant.e4m3_round(x.astype(np.float32).astype(np.float64)), ref)


def test_e4m3_saturates_and_keeps_representable():
    assert quant.e4m3_round(np.array([1000.0, -1e6]))[0] == 448.0
    assert np.array_equal(quant.e4m3_round(quant._E4M3), quant._E4M3)


def test_fp8_sketch_scales_and_structure():
    from oracle import sketch

    A = np.random.default_rng(4).standard_normal((300, 6)).astype(np.float32)
    A[:, 2] = 0.0
    s, r = sketch.fp8_column_scales(A)
    assert s[2] == 1.0 and np.all(np.abs(A * r[None, :]) <= 448.0 * (1 + 2 ** -20))
    # E4M3 keeps 3 mantissa bits (relative rounding error <= 2^-4 per operand), so
    # the quantised sketch stays close to the unquantised one
    got = sketch.gaussian_sketch_fp8(A, 5, 1, 0)
    ref = sketch.gaussian_sketch(A, 5, 1, 0)
    assert np.linalg.norm(got - ref) <= 0.1 * np.linalg.norm(ref)


def _z32(m, n, seed, level):
    from oracle import rng

    return rng.gaussian_z_cols(m, 0, n, seed, level).astype(np.float32)


def test_bf16_sketch_of_identity_is_rounded_z():
    """A = I_n: the BF16 sketch is bf16(fl32(z)) / sqrt(m) entry by entry, with
    the rounding done by torch's CPU cast of the binary32 draws (a library,
    independent of the oracle).  Dropping the rounding of z, or rounding z from
    its float64 value instead of binary32, changes some entries."""
    from oracle import rng, sketch

    m, n, seed, level = 48, 8192, 3, 5
    got = sketch.gaussian_sketch_bf16(np.eye(n, dtype=np.float32), m, seed, level, block=2048)
    z32 = _z32(m, n, seed, level)
    expect = torch.from_numpy(z32).to(torch.bfloat16).to(torch.float64).numpy() / np.sqrt(m)
    assert np.array_equal(got, expect)
    # the input has the power to tell the two plausible mistakes apart
    z64 = rng.gaussian_z_cols(m, 0, n, seed, level)
    unrounded = z32.astype(np.float64) / np.sqrt(m)
    assert not np.array_equal(got, unrounded)
    # float64 z rounded once to 8 significant bits (ties to even): differs from
    # the binary32-first rounding where the binary32 step lands on a midpoint
    mant, ex = np.frexp(z64)
    from_f64 = np.ldexp(np.round(mant * 256.0) / 256.0, ex) / np.sqrt(m)
    assert np.count_nonzero(from_f64 != expect) >= 1


def test_fp8_sketch_of_scaled_identity_pairs():
    """A with two non-zeros per column, a_{i,i} = c_i and a_{n/2+i,i} = c_i v_i:
    column i of the E4M3 sketch is
    (e4m3(z_{j,i}) e4m3(fl32(c_i r_i)) + e4m3(z_{j,n/2+i}) e4m3(fl32(c_i v_i r_i))) s_i / sqrt(m),
    s_i = fl32(c_i / 448), r_i = fl32(1 / s_i), every rounding by torch's CPU
    cast.  Both products and their sum are exact in float64, so the comparison
    is exact: a dropped diag(s), r in place of s, or an unrounded z all fail."""
    from oracle import sketch

    g = np.random.default_rng(7)
    half, m, seed, level = 512, 24, 2, 3
    n = 2 * half
    c = (10.0 ** g.uniform(-3, 3, half)).astype(np.float32)
    v = g.uniform(0.01, 0.99, half).astype(np.float32)
    A = np.zeros((n, half), dtype=np.float32)
    A[np.arange(half), np.arange(half)] = c
    A[half + np.arange(half), np.arange(half)] = (c * v).astype(np.float32)
    got = sketch.gaussian_sketch_fp8(A, m, seed, level, block=256)

    def q(x32):
        return torch.from_numpy(np.ascontiguousarray(x32)).to(torch.float8_e4m3fn).to(torch.float64).numpy()

    s = (c / np.float32(448.0)).astype(np.float32)
    r = (np.float32(1.0) / s).astype(np.float32)
    z = _z32(m, n, seed, level)
    top = q((c * r).astype(np.float32))
    bot = q(((c * v).astype(np.float32) * r).astype(np.float32))
    expect = (q(z[:, :half]) * top[None, :] + q(z[:, half:]) * bot[None, :]) * s.astype(np.float64)[None, :] / np.sqrt(m)
    assert np.array_equal(got, expect)
    assert not np.allclose(s, r)   # s and r are far apart: swapping them would fail
