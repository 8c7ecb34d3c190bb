"""The bounds' quotients are formed as q0 = x r, q = q0 + (x - q0 c) r with
r = RN(1/c) and two fused multiply-adds (Markstein's correction step, IBM J.
Res. Dev. 34 (1990) 111): the correctly rounded quotient RN(x/c), the IEEE
division's value, for finite x whose quotient is normal.  Here the two FMAs
are evaluated exactly (rational arithmetic, one rounding each), for the
divisors the step uses: sigma_max = 400, the temperature bound 100, and the
beta bound's 2 (gamma - 1) for the adiabatic indices of the test problems.
Against Python's float division, which rounds correctly."""
import random
from fractions import Fraction

import pytest


def _rn(fr):
    return fr.numerator / fr.denominator  # int / int rounds correctly


def _fma(a, b, c):
    return _rn(Fraction(a) * Fraction(b) + Fraction(c))


def _div_rn(x, c, rc):
    q0 = x * rc
    r = _fma(-q0, c, x)
    return _fma(r, rc, q0)


DIVISORS = [400.0, 100.0] + [2.0 * (g - 1.0) for g in (4.0 / 3.0, 5.0 / 3.0, 1.4, 13.0 / 9.0)]


@pytest.mark.parametrize("c", DIVISORS)
def test_correction_step_is_the_ieee_quotient(c):
    rc = 1.0 / c
    rng = random.Random(int(c * 1e6))
    xs = [(rng.getrandbits(52) | (1 << 52)) * 2.0 ** (rng.randint(-300, 300) - 52)
          for _ in range(15000)]
    # significands at and beside powers of two, and multiples of the divisor
    for e in range(-200, 201, 40):
        p = 2.0 ** e
        xs += [p, p * (1 + 2.0 ** -52), p * (2 - 2.0 ** -52), p * c, p * c * (1 + 2.0 ** -52)]
    bad = [x for x in xs if _div_rn(x, c, rc) != x / c]
    assert not bad, (c, bad[:3])


def test_plain_product_is_not():
    """The reciprocal's product alone, RN(x RN(1/c)), misses the IEEE quotient
    in a fair share of cases: the correction step is doing the work."""
    rng = random.Random(3)
    xs = [rng.uniform(1.0, 2.0) for _ in range(2000)]
    miss = sum(1 for x in xs if x * (1.0 / 400.0) != x / 400.0)
    assert miss > 100
