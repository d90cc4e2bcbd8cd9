"""The arithmetic premise of the tensor-core Gram (App. B.4's K = nu^2 I + SA SA^T
formed from binary32 SA): every binary32 x equals p1 + p2 + p3 with
p1 = bf16(x), p2 = bf16(x - p1), p3 = bf16(x - p1 - p2) (round to nearest even,
the residuals formed in binary32), and a product of two BF16 pieces is exact in
binary32, so x_a x_b is the exact sum of the nine piece-pair products.  BF16
rounding is emulated here with integer operations on the bit patterns."""
import numpy as np


def bf16_rn(x):
    """Round binary32 values to BF16 (8 significant bits), nearest even."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = (u + 0x7FFF + lsb) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def split3(x):
    x = np.asarray(x, dtype=np.float32)
    p1 = bf16_rn(x)
    r1 = (x - p1).astype(np.float32)
    p2 = bf16_rn(r1)
    r2 = (r1 - p2).astype(np.float32)
    p3 = bf16_rn(r2)
    return p1, p2, p3, r2


def _samples():
    g = np.random.default_rng(7)
    xs = [g.standard_normal(200000).astype(np.float32) * s for s in (1.0, 1e-3, 1.0 / 45.0, 3e4)]
    special = np.array([1.0, -1.0, 2.0 ** -100, 1.0 + 2.0 ** -23, 1.0 - 2.0 ** -24, 3.0, 255.5, 1e30,
                        np.float32(np.pi), -np.float32(np.e)], dtype=np.float32)
    return np.concatenate(xs + [special])


def test_three_pieces_reconstruct_exactly():
    x = _samples()
    p1, p2, p3, r2 = split3(x)
    assert np.array_equal(p3, r2)   # the last residual already fits in BF16
    total = p1.astype(np.float64) + p2.astype(np.float64) + p3.astype(np.float64)
    assert np.array_equal(total, x.astype(np.float64))
    for p in (p1, p2, p3):          # each piece has at most 8 significant bits
        assert np.array_equal(bf16_rn(p), p)


def test_piece_products_exact_in_binary32():
    g = np.random.default_rng(8)
    a = (g.standard_normal(50000) / 45.0).astype(np.float32)
    b = (g.standard_normal(50000) / 45.0).astype(np.float32)
    pa, pb = split3(a)[:3], split3(b)[:3]
    exact = a.astype(np.float64) * b.astype(np.float64)
    acc = np.zeros_like(exact)
    for u in pa:
        for v in pb:
            prod32 = (u * v).astype(np.float32)
            assert np.array_equal(prod32.astype(np.float64), u.astype(np.float64) * v.astype(np.float64))
            acc += prod32.astype(np.float64)
    assert np.allclose(acc, exact, rtol=0, atol=0)


def test_a_dropped_piece_would_be_caught():
    # two pieces do not suffice: the premise needs the third
    x = _samples()
    p1, p2, _, _ = split3(x)
    two = p1.astype(np.float64) + p2.astype(np.float64)
    assert not np.array_equal(two, x.astype(np.float64))
