"""Pins of the oracle's reconstruction.

* MC: exact on linear data, zero slope at an extremum, the limited slope of
  a worked case by hand.
* WENO5 (Jiang-Shu): exact on quadratics (every candidate stencil is), a
  face value of smooth data converges at fifth order, and the left/right
  values mirror each other.
"""
import math

import numpy as np
import pytest

import oracle


def test_mc_linear_exact():
    l, r = oracle.recon(0, [1.0, 3.0, 5.0])
    assert (l, r) == (2.0, 4.0)


def test_mc_extremum_flat():
    assert oracle.recon(0, [1.0, 3.0, 2.0]) == (3.0, 3.0)
    assert oracle.recon(0, [3.0, 1.0, 2.0]) == (1.0, 1.0)


def test_mc_limited_by_hand():
    # dm = 1, dp = 4, centred 2.5: min(2, 2.5, 8) = 2 -> faces 0 and 2
    assert oracle.recon(0, [0.0, 1.0, 5.0]) == (0.0, 2.0)
    # dm = -4, dp = -1: min(8, 2.5, 2) = 2, negative slope
    assert oracle.recon(0, [5.0, 1.0, 0.0]) == (2.0, 0.0)


@pytest.mark.parametrize("coef", [(0.3, -1.2, 0.7), (2.0, 0.0, -3.0), (-1.0, 5.0, 0.25)])
def test_weno5_quadratic_exact(coef):
    """Zone values are cell averages of a quadratic (Jiang-Shu's
    finite-volume form): the face values are the quadratic at the faces."""
    c0, c1, c2 = coef
    f = lambda x: c0 + c1 * x + c2 * x * x
    xs = np.arange(-2, 3) * 0.1 + 0.37
    avg = f(xs) + c2 * 0.1 ** 2 / 12.0
    l, r = oracle.recon(1, avg)
    assert l == pytest.approx(f(0.37 - 0.05), rel=1e-12, abs=1e-13)
    assert r == pytest.approx(f(0.37 + 0.05), rel=1e-12, abs=1e-13)


def test_weno5_fifth_order():
    errs = []
    for h in (0.2, 0.1, 0.05):
        x0 = 0.3
        xs = x0 + np.arange(-2, 3) * h
        avg = (np.cos(xs - h / 2) - np.cos(xs + h / 2)) / h
        l, r = oracle.recon(1, avg)
        errs.append(abs(r - math.sin(x0 + h / 2)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 4.3), (errs, orders)


def test_weno5_mirror():
    x = np.array([0.1, -0.4, 2.0, 1.1, 0.9])
    l, r = oracle.recon(1, x)
    l2, r2 = oracle.recon(1, x[::-1])
    assert l == r2 and r == l2


def test_weno5_nonoscillatory_at_jump():
    """At a step the face values stay within the data range."""
    l, r = oracle.recon(1, [0.0, 0.0, 0.0, 1.0, 1.0])
    assert -1e-6 <= l <= 1e-6 and 0.0 <= r <= 1.0
    assert r < 0.1


def test_weno5_zone_pair_equals_single_face_form():
    """The step reconstructs each zone's two faces from one set of
    smoothness indicators; each value equals the single-face form (each
    face from its own indicators, the mirrored stencil for the low face)
    to rounding, on smooth data, steps, extrema and constants."""
    rng = np.random.default_rng(11)
    cases = [rng.normal(size=5) for _ in range(300)]
    cases += [np.where(np.arange(5) < k, 1.0, 0.0) * rng.uniform(1, 10) for k in range(1, 5)]
    cases += [np.full(5, 3.0), np.array([0, 1, 4, 1, 0.0]), np.array([1e-30, 2e-30, 0, 5e-31, 1e-30])]
    for x in cases:
        z = oracle.recon(oracle.RECON_WENO5 if hasattr(oracle, "RECON_WENO5") else 1, x)
        f = oracle.recon_faces(x)
        scale = np.abs(x).max()
        assert np.abs(z - f).max() <= 1e-14 * max(scale, 1e-300), (x, z, f)
