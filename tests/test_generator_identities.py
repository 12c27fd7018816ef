"""CPU checks of the exact floating-point identities the FP32 generator's
device code relies on (the device then needs no separate proof):

* the uniform u = (2k + 1) 2^-24 of a 23-bit k equals (1 + k 2^-23) minus
  (1 - 2^-24) in one FP32 subtraction, for every k;
* scaling a round-to-nearest FP32 operation's operands by -2 scales its
  result by -2 (no overflow or underflow on the LOG's range), so the LOG
  with every constant multiplied by -2 returns -2 LOG(u) bit for bit;
* negation is the sign bit (sign flips as bit flips)."""
import numpy as np


def test_uniform_by_one_subtraction_is_exact():
    k = np.arange(1 << 23, dtype=np.uint32)
    one_plus = (np.uint32(0x3F800000) | k).view(np.float32)
    got = one_plus - np.float32(1.0 - 2.0 ** -24)
    want = ((2 * k.astype(np.float64) + 1) * 2.0 ** -24).astype(np.float32)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_minus_two_scaling_commutes_with_rounding():
    # every step of the FP32 LOG is an IEEE add, multiply or fma; for
    # products and sums, RN(-2 x) = -2 RN(x) while no value leaves the
    # normal range: the LOG's intermediates lie within [2^-50, 2^7]
    rng = np.random.default_rng(0)
    a = rng.uniform(-4, 4, 1 << 20).astype(np.float32)
    b = rng.uniform(-4, 4, 1 << 20).astype(np.float32)
    m2 = np.float32(-2.0)
    assert np.array_equal((m2 * a) * b, m2 * (a * b))
    assert np.array_equal((m2 * a) + (m2 * b), m2 * (a + b))
    # a fused multiply-add rounds once, like the sum above (emulated exactly
    # in FP64 for operands whose product and sum fit 53 bits)
    c = rng.uniform(-4, 4, 1 << 20).astype(np.float32)
    fma = lambda x, y, z: (x.astype(np.float64) * y + z).astype(np.float32)
    a16 = a.astype(np.float16).astype(np.float32)   # 11-bit operands: the FP64 sum is exact
    b16 = b.astype(np.float16).astype(np.float32)
    c16 = c.astype(np.float16).astype(np.float32)
    assert np.array_equal(fma(m2 * a16, b16, m2 * c16), m2 * fma(a16, b16, c16))


def test_negation_is_the_sign_bit():
    x = np.random.default_rng(1).standard_normal(1 << 16).astype(np.float32)
    x[:4] = [0.0, -0.0, np.inf, -np.inf]
    assert np.array_equal((-x).view(np.uint32), x.view(np.uint32) ^ np.uint32(0x80000000))
