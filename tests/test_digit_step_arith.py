"""CPU check of the arithmetic identity behind the split path's digit step.

The digit kernels take balanced base-2^LB digits of a normalised double-float (xh, xl):
d = rint(xh), a = xh - d, then Fast2Sum(a, xl) = (s, e) re-joins the remainder exactly and
both parts are scaled by 2^LB for the next digit.  The packed kernel folds the scaling into
the Fast2Sum: 2^LB s = RN(2^LB a + 2^LB xl) is one FMA, and the FMA 2^LB s - 2^LB a returns
2^LB (s - a) unrounded, so 2^LB xl minus it is the error term 2^LB e.  This test emulates
both sequences in IEEE binary32 (round to nearest even; the FMA rounded once from the exact
rational value) and checks that they give the same digits and remainders bit for bit.
"""
from fractions import Fraction

import numpy as np
import pytest

f32 = np.float32
SHIFT = f32(12582912.0)   # 1.5 * 2^23: (x + SHIFT) - SHIFT = rint(x) for |x| <= 2^22


def round_f32(q: Fraction) -> np.float32:
    """The binary32 value nearest to the rational q (ties to even), gradual underflow."""
    if q == 0:
        return f32(0.0)
    sign = -1 if q < 0 else 1
    q = abs(q)
    e = q.numerator.bit_length() - q.denominator.bit_length()
    if Fraction(2) ** e > q:
        e -= 1
    e = max(e, -126)                       # subnormals share the exponent of 2^-126
    scale = Fraction(2) ** (23 - e)
    m = q * scale
    fl = m.numerator // m.denominator
    rem = m - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    val = Fraction(fl) / scale
    assert val < Fraction(2) ** 128, "overflow is outside the tested range"
    return f32(sign * float(val))          # exact: val has at most 24 significant bits


def fma32(a, b, c) -> np.float32:
    return round_f32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def step_fast2sum(xh, xl, lb):
    """The scalar digit step: rint, remainder, Fast2Sum, scaling."""
    sc = f32(2.0 ** lb)
    d = (xh + SHIFT) - SHIFT
    a = xh - d
    s = a + xl
    e = xl - (s - a)
    return d, s * sc, e * sc


def step_fma(xh, xl, lb):
    """The packed kernel's digit step with the scaling folded into FMAs."""
    sc = f32(2.0 ** lb)
    d = (xh + SHIFT) - SHIFT
    a = xh - d
    l = xl * sc
    nh = fma32(a, sc, l)
    nl = l - fma32(a, -sc, nh)
    return d, nh, nl


def normalised_pair(rng, bound):
    """(xh, xl) with xh = RN(x) and xl = RN(x - xh) for a random x, so |xl| <= ulp(xh)/2."""
    x = rng.uniform(-bound, bound) * 2.0 ** -int(rng.integers(0, 30))
    xh = f32(x)
    xl = f32(x - float(xh))
    return xh, xl


def special_pairs(bound):
    pairs = [(f32(0.0), f32(0.0)), (f32(0.5), f32(0.0)), (f32(-0.5), f32(0.0)),
             (f32(1.5), f32(0.0)), (f32(2.5), f32(0.0)), (f32(bound), f32(0.0)),
             (f32(-bound), f32(0.0))]
    for base in (0.5, 1.5, -2.5, 3.5, bound - 0.5):
        h = f32(base)
        u = float(np.spacing(h))
        pairs += [(h, f32(u / 2)), (h, f32(-u / 2)), (h, f32(u / 4))]
    return pairs


@pytest.mark.parametrize("lb,bound,planes", [(9, 64.0, 6), (5, 16.0, 10)])
def test_fma_folded_digit_step_is_bit_identical(lb, bound, planes):
    rng = np.random.default_rng(1234 + lb)
    cases = special_pairs(bound) + [normalised_pair(rng, bound) for _ in range(400)]
    for xh0, xl0 in cases:
        h1, l1 = xh0, xl0
        h2, l2 = xh0, xl0
        for _ in range(planes):
            d1, h1, l1 = step_fast2sum(h1, l1, lb)
            d2, h2, l2 = step_fma(h2, l2, lb)
            assert d1.tobytes() == d2.tobytes()
            assert h1.tobytes() == h2.tobytes() and l1.tobytes() == l2.tobytes()
            assert abs(float(d1)) <= 2.0 ** (lb - 1)


def test_round_f32_matches_numpy_on_doubles():
    # the FMA emulation's rounding agrees with numpy's float64 -> float32 conversion
    # wherever the input is a double (single rounding from an exact value)
    rng = np.random.default_rng(7)
    for x in rng.standard_normal(300) * 10.0 ** rng.integers(-20, 20, 300):
        assert round_f32(Fraction(float(x))).tobytes() == f32(x).tobytes()
