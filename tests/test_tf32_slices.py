"""Number formats of the mixed path's tensor-core operands, checked in numpy
(independent of the library): TF32 rounding to nearest with ties away from
zero (10 stored mantissa bits), the two-piece split x = hi + lo of the
3xTF32 products, and the four slices h + m + q + s of the reference block
F0 that the fused energy contraction adds through identity blocks of its A
operand (one slice pair per identity block).
"""
import numpy as np


def tf32(x):
    """Round FP32 values to TF32 (nearest, ties away from zero)."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    sign = b & 0x80000000
    mag = b & 0x7FFFFFFF
    mag = (mag + 0x1000) & 0x7FFFE000          # add half an ulp of the 10-bit mantissa, truncate
    return (sign | mag).astype(np.uint32).view(np.float32)


def slices4(x):
    """h = tf32(x), m = tf32(x - h), q = tf32(x - h - m), s = tf32(x - h - m - q), remainders in FP64."""
    out = []
    v = np.asarray(x, dtype=np.float64)
    for _ in range(4):
        p = tf32(v.astype(np.float32))
        out.append(p)
        v = v - p.astype(np.float64)
    return out, v


def test_tf32_rounding_keeps_eleven_significant_bits():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(100000) * np.exp(rng.uniform(-20, 20, 100000))).astype(np.float32)
    r = tf32(x)
    # exactly representable in 11 significant bits
    m, _ = np.frexp(r.astype(np.float64))
    assert np.all(np.abs(m * 2.0 ** 11 - np.round(m * 2.0 ** 11)) == 0)
    # round to nearest: error at most half a TF32 ulp (2^-11 relative to the binade)
    err = np.abs(r.astype(np.float64) - x.astype(np.float64))
    _, e = np.frexp(x.astype(np.float64))
    assert np.all(err <= 2.0 ** (e.astype(np.float64) - 12))
    # ties go away from zero
    t = np.array([1.0 + 2.0 ** -11, -(1.0 + 2.0 ** -11), 1.0 + 3 * 2.0 ** -11], dtype=np.float32)
    assert list(tf32(t)) == [np.float32(1.0 + 2.0 ** -10), np.float32(-(1.0 + 2.0 ** -10)),
                             np.float32(1.0 + 2.0 ** -9)]


def test_four_slices_represent_f0_to_about_44_bits():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(200000) * np.exp(rng.uniform(-8, 8, 200000))
    sl, rem = slices4(x)
    total = sum(p.astype(np.float64) for p in sl)
    assert np.all(np.abs(x - total) == np.abs(rem))
    assert np.max(np.abs(rem) / np.abs(x)) < 2.0 ** -42
    # each slice is a TF32 value, so the tensor cores take it without loss
    for p in sl:
        assert np.array_equal(tf32(p), p)
    # two slices (one identity block) would leave about 2^-22
    two = (sl[0].astype(np.float64) + sl[1].astype(np.float64))
    assert np.max(np.abs(x - two) / np.abs(x)) > 2.0 ** -26


def test_identity_blocks_reproduce_f0_through_three_products():
    """An identity column block of A (hi = 1, lo = 0) against B slices
    (hi, lo) contributes a_hi b_hi + a_hi b_lo + a_lo b_hi = b_hi + b_lo: two
    blocks with (h, m) and (q, s) give h + m + q + s on the real-part rows
    and nothing on the imaginary-part rows (their identity blocks are zero)."""
    rng = np.random.default_rng(2)
    N, RB, ncol = 5, 8, 7
    F0 = rng.standard_normal((N, ncol))
    (h, m, q, s), _ = slices4(F0)
    # A rows (c, j), K columns [block 1 | block 2], each RB wide
    a_hi = np.zeros((2, RB, 2 * RB))
    for j in range(N):
        a_hi[0, j, j] = a_hi[0, j, RB + j] = 1.0
    a_lo = np.zeros_like(a_hi)
    b_hi = np.zeros((ncol, 2 * RB))
    b_lo = np.zeros((ncol, 2 * RB))
    b_hi[:, :N], b_lo[:, :N] = h.T, m.T
    b_hi[:, RB:RB + N], b_lo[:, RB:RB + N] = q.T, s.T
    D = a_hi @ b_hi.T + a_hi @ b_lo.T + a_lo @ b_hi.T
    assert np.max(np.abs(D[0, :N] - F0)) < 2.0 ** -42 * np.max(np.abs(F0))
    assert np.all(D[1] == 0) and np.all(D[0, N:] == 0)
