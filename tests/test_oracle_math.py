"""Pins for the oracle's own elementary functions and their constants.

The scenario generator turns Philox words into normals by Box-Muller and into
lognormal innovations by exp; both sides of the parity check implement LOG,
SIN2PI/COS2PI and EXP themselves so that samples agree bit for bit.  Here the
oracle's versions are held to ulp bounds against numpy/mpmath, exhaustively
over every float32 uniform the generator can produce, and every constant is
checked to be the correctly rounded value of its definition.
"""
import mpmath
import numpy as np
import pytest

import oracle

mpmath.mp.prec = 200


def _rn(x, bits):
    old = mpmath.mp.prec
    mpmath.mp.prec = bits
    y = +mpmath.mpf(x)
    mpmath.mp.prec = old
    return float(y)


def _ulp32(x):
    return np.spacing(np.abs(x).astype(np.float32)).astype(np.float64)


LN2 = mpmath.log(2)


@pytest.mark.parametrize("bits,which_s", [(24, 0), (53, 1)])
def test_scalar_constants_correctly_rounded(bits, which_s):
    hi = _rn(LN2, 16 if bits == 24 else 32)
    exact = [mpmath.sqrt(2), mpmath.mpf(hi), LN2 - mpmath.mpf(hi), 1 / LN2, mpmath.e ** mpmath.mpf("0.5"),
             1 / mpmath.sqrt(mpmath.e ** 2 - mpmath.e)]
    got = oracle.constants(which_s)
    want = [_rn(v, bits) for v in exact]
    assert list(got) == want


@pytest.mark.parametrize("which,bits,term", [
    (2, 24, lambda k: mpmath.mpf(2) / (2 * k + 1)),
    (3, 53, lambda k: mpmath.mpf(2) / (2 * k + 1)),
    (4, 24, lambda k: (-1) ** k * (2 * mpmath.pi) ** (2 * k + 1) / mpmath.factorial(2 * k + 1)),
    (5, 53, lambda k: (-1) ** k * (2 * mpmath.pi) ** (2 * k + 1) / mpmath.factorial(2 * k + 1)),
    (6, 24, lambda k: (-1) ** k * (2 * mpmath.pi) ** (2 * k) / mpmath.factorial(2 * k)),
    (7, 53, lambda k: (-1) ** k * (2 * mpmath.pi) ** (2 * k) / mpmath.factorial(2 * k)),
    (8, 24, lambda k: 1 / mpmath.factorial(k)),
    (9, 53, lambda k: 1 / mpmath.factorial(k)),
])
def test_series_coefficients_correctly_rounded(which, bits, term):
    got = oracle.constants(which)
    want = [_rn(term(k), bits) for k in range(len(got))]
    assert list(got) == want


# every uniform the float generator produces: u = n 2^-24, n odd in [1, 2^24)
_N24 = np.arange(1, 1 << 24, 2, dtype=np.uint32)
_U24 = (_N24.astype(np.float64) * 2.0 ** -24).astype(np.float32)


def test_log_f32_exhaustive_within_3ulp():
    got = oracle.log_f32(_U24).astype(np.float64)
    ref = np.log(_U24.astype(np.float64))
    err = np.abs(got - ref) / _ulp32(ref)
    assert err.max() <= 3.0


def test_sincos2pi_f32_exhaustive_within_2ulp():
    s, c = oracle.sincos2pi_f32(_N24)
    a = 2.0 * np.pi * _U24.astype(np.float64)
    rs, rc = np.sin(a), np.cos(a)
    assert (np.abs(s - rs) / _ulp32(rs)).max() <= 2.0
    assert (np.abs(c - rc) / _ulp32(rc)).max() <= 2.0
    # the quadrant rotation keeps sin^2 + cos^2 = 1 to float rounding
    r2 = s.astype(np.float64) ** 2 + c.astype(np.float64) ** 2
    assert np.abs(r2 - 1.0).max() < 4e-7


def test_exp_f32_within_1ulp_on_box_muller_range():
    x = np.linspace(-7.0, 7.0, 2_000_001).astype(np.float32)
    got = oracle.exp_f32(x).astype(np.float64)
    ref = np.exp(x.astype(np.float64))
    assert (np.abs(got - ref) / _ulp32(ref)).max() <= 1.0


def _u53_samples(n, seed):
    rng = np.random.default_rng(seed)
    nums = 2 * rng.integers(0, 2 ** 52, size=n, dtype=np.uint64) + 1
    nums[:4] = np.array([1, 3, 2 ** 53 - 1, 2 ** 52 + 1], dtype=np.uint64)
    return nums.astype(np.uint64)


def test_log_f64_within_2ulp():
    nums = _u53_samples(3000, 11)
    u = nums.astype(np.float64) * 2.0 ** -53
    got = oracle.log_f64(u)
    ref = np.array([float(mpmath.log(mpmath.mpf(int(n)) * mpmath.mpf(2) ** -53)) for n in nums])
    assert (np.abs(got - ref) / np.spacing(np.abs(ref))).max() <= 2.0


def test_sincos2pi_f64_within_1ulp():
    nums = _u53_samples(3000, 12)
    s, c = oracle.sincos2pi_f64(nums)
    ang = [2 * mpmath.pi * mpmath.mpf(int(n)) * mpmath.mpf(2) ** -53 for n in nums]
    rs = np.array([float(mpmath.sin(a)) for a in ang])
    rc = np.array([float(mpmath.cos(a)) for a in ang])
    assert (np.abs(s - rs) / np.spacing(np.abs(rs))).max() <= 1.0
    assert (np.abs(c - rc) / np.spacing(np.abs(rc))).max() <= 1.0


def test_exp_f64_within_1ulp():
    x = np.random.default_rng(13).uniform(-8.0, 8.0, 3000)
    got = oracle.exp_f64(x)
    ref = np.array([float(mpmath.exp(mpmath.mpf(v))) for v in x])
    assert (np.abs(got - ref) / np.spacing(ref)).max() <= 1.0
