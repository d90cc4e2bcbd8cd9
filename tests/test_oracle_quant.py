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
    # with every operand exactly representable the quantised sketch is the sketch
    got = sketch.gaussian_sketch_fp8(A, 5, 1, 0)
    ref = sketch.gaussian_sketch(A, 5, 1, 0)
    assert np.linalg.norm(got - ref) <= 0.1 * np.linalg.norm(ref)
