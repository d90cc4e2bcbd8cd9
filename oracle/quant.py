"""Rounding to the low-precision operand formats the tensor-core sketch uses.

* BF16: IEEE binary32 with the low 16 bits rounded away, round to nearest,
  ties to even.
* FP8 E4M3 (the "fn" variant: no infinities, max finite 448): 1 sign bit, 4
  exponent bits (bias 7), 3 mantissa bits; round to nearest, ties to even,
  saturating at +-448.

The Gaussian sketch with low-precision operands computes
SA = diag(1 / sqrt(m)) q(Z) q(A) exactly apart from FP32 accumulation, q the
rounding above (with per-column scales for FP8).  Pinned against torch's CPU
conversions in tests/test_oracle_quant.py.
"""
import numpy as np


def bf16_round(x):
    """Round float32 values to the nearest bfloat16 (ties to even); returns float32."""
    x = np.asarray(x, dtype=np.float32)
    bits = x.view(np.uint32).astype(np.uint64)
    lsb = (bits >> np.uint64(16)) & np.uint64(1)
    rounded = ((bits + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return (rounded & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)


def _e4m3_values():
    vals = [0.0]
    for e in range(16):
        for mant in range(8):
            if e == 15 and mant == 7:
                continue          # NaN encoding
            if e == 0:
                v = mant / 8.0 * 2.0 ** -6
            else:
                v = (1.0 + mant / 8.0) * 2.0 ** (e - 7)
            vals.append(v)
    vals = np.array(sorted(set(vals)), dtype=np.float64)
    return vals


_E4M3 = _e4m3_values()   # non-negative finite values, ascending; max 448
# the mantissa LSB of each value (for ties to even): index parity in the code order
_E4M3_CODE = {v: i for i, v in enumerate(_E4M3)}


def e4m3_round(x):
    """Round to the nearest FP8 E4M3 value (ties to even, saturating); float64 out."""
    x = np.asarray(x, dtype=np.float64)
    a = np.minimum(np.abs(x), _E4M3[-1])
    hi = np.searchsorted(_E4M3, a, side="left")
    hi = np.clip(hi, 0, len(_E4M3) - 1)
    lo = np.clip(hi - 1, 0, len(_E4M3) - 1)
    vlo, vhi = _E4M3[lo], _E4M3[hi]
    dlo, dhi = a - vlo, vhi - a
    # consecutive codes alternate mantissa parity; the even code has an even index
    pick_hi = (dhi < dlo) | ((dhi == dlo) & (hi % 2 == 0))
    r = np.where(pick_hi, vhi, vlo)
    r = np.where(a == vhi, vhi, r)
    return np.sign(x) * r
