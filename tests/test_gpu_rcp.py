"""The reciprocal, reciprocal square root and square root the step uses
inside its arithmetic (WENO5 weights, fluid states, signal speeds, the
Newton iteration of the 1D_W inversion): hardware approximations refined by
one step of a series (the geometric series of 1/(1 - e) for the
reciprocal, the binomial series of (1 - h)^(-1/2) for the reciprocal square
root; the square root is x times the latter).  Against the IEEE results
computed on the same device (torch's reciprocal, rsqrt and sqrt), each must
be within 2 ulp over the normal range it is specified for: values spread
log-uniformly over 1e-300 .. 1e300 (both signs for the reciprocal), the
magnitudes the WENO5 pair feeds the reciprocal (products of two sums of
squared smoothness indicators), 1 + q^2 and 1 - v^2 as the fluid state and
the inversion form them, and exact powers of two.  Outside
[2^-1022, 2^1022] the reciprocal flushes (zero or subnormal x -> NaN,
|x| > 2^1022 -> 0), as the header states.  The bounds' quotients (one
correction step from the divisor's reciprocal) must equal the device's IEEE
division bit for bit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2110_10191_gb300 import grmhd
    grmhd.load()
    return torch, grmhd


def _ulps(a, b):
    """Distance in units in the last place between float64 arrays of one sign."""
    ia = a.view(np.int64)
    ib = b.view(np.int64)
    return np.abs(ia - ib)


def _weno_denominators(rng, n):
    """H L of the WENO5 pair for random 5-zone stencils whose values span
    1e-12 .. 1e3 (densities at the floor up to large field energies): H and
    L are sums of products of two squared 4 eps + 4 beta_k, with 4 beta_k =
    (13/3) D_k^2 + s_k^2 from the stencil's first and second differences."""
    scale = 10.0 ** rng.uniform(-12, 3, n)
    a, b, c, d, e = 1.0 + rng.standard_normal((5, n)) * 10.0 ** rng.uniform(-8, 0, n)
    a, b, c, d, e = a * scale, b * scale, c * scale, d * scale, e * scale
    dm2, dm1, dp1, dp2 = b - a, c - b, d - c, e - d
    D0, D1, D2 = dm1 - dm2, dp1 - dm1, dp2 - dp1
    s0, s1, s2 = D0 + 2 * dm1, dm1 + dp1, D2 - 2 * dp1
    q0, q1, q2 = [(4e-26 + (13 / 3) * D * D + s * s) ** 2 for D, s in ((D0, s0), (D1, s1), (D2, s2))]
    H = q1 * q2 + 6 * q0 * q2 + 3 * q0 * q1
    L = q0 * q1 + 6 * q0 * q2 + 3 * q1 * q2
    return H * L


def _run(dev, fn, xs):
    torch, grmhd = dev
    x = torch.from_numpy(xs).cuda()
    out = torch.empty_like(x)
    grmhd.arith(fn, x, out)
    refs = {"rcp": torch.reciprocal, "rsqrt": torch.rsqrt, "sqrt": torch.sqrt}
    ref = refs[fn](x) if fn in refs else None
    torch.cuda.synchronize()
    return out.cpu().numpy(), None if ref is None else ref.cpu().numpy()


def _normal(xs):
    return xs[np.isfinite(xs) & (np.abs(xs) >= 2.0 ** -1022) & (np.abs(xs) <= 2.0 ** 1022)]


def test_rcp_within_2_ulp_of_ieee_division(dev):
    rng = np.random.default_rng(7)
    n = 1 << 20
    mag = 10.0 ** rng.uniform(-300, 300, n)
    sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    pows = 2.0 ** np.arange(-1022, 1023, dtype=np.float64)
    xs = _normal(np.concatenate([mag * sign, _weno_denominators(rng, n // 4), pows, -pows,
                                 np.nextafter(pows, 0.0)[1:], 1.0 + np.arange(1, 4096) * 2.0 ** -52]))
    a, b = _run(dev, "rcp", xs)
    assert np.all(np.sign(a) == np.sign(b))
    u = _ulps(a, b)
    assert u.max() <= 2, (int(u.max()), float(xs[int(np.argmax(u))]))
    # and most are exact: the third-order step leaves ~2^-60 before rounding
    assert (u == 0).mean() > 0.9


@pytest.mark.parametrize("fn", ["rsqrt", "sqrt"])
def test_rsqrt_and_sqrt_within_2_ulp_of_ieee(dev, fn):
    rng = np.random.default_rng(11)
    n = 1 << 20
    mag = 10.0 ** rng.uniform(-300, 300, n)
    pows = 2.0 ** np.arange(-1022, 1023, dtype=np.float64)
    # 1 + q^2 of the fluid state (q up to a Lorentz factor of ~1e3) and
    # 1 - v^2 of the inversion (down to its limit 1e-10)
    lorentz = 1.0 + (10.0 ** rng.uniform(-12, 3, n // 4)) ** 2
    omv = 1.0 - (1.0 - 10.0 ** rng.uniform(-10, 0, n // 4))
    xs = _normal(np.concatenate([mag, _weno_denominators(rng, n // 8), lorentz, omv, pows,
                                 np.nextafter(pows, np.inf)[:-1]]))
    a, b = _run(dev, fn, xs)
    assert np.all(a > 0)
    u = _ulps(a, b)
    assert u.max() <= 2, (int(u.max()), float(xs[int(np.argmax(u))]))
    assert (u == 0).mean() > 0.5


def test_rcp_outside_the_normal_range(dev):
    """The approximation flushes subnormal inputs and results to zero: a
    zero or subnormal x gives NaN (the refinement meets inf * 0), |x| above
    2^1022 (a subnormal quotient) gives a zero of x's sign."""
    torch, grmhd = dev
    xs = np.array([2.0 ** -1074, -2.0 ** -1040, 0.0, 2.0 ** 1022 * 1.5, -(2.0 ** 1023)])
    a, _ = _run(dev, "rcp", xs)
    assert np.all(np.isnan(a[:3]))
    assert a[3] == 0.0 and not np.signbit(a[3])
    assert a[4] == 0.0 and np.signbit(a[4])
    with pytest.raises(grmhd.GrmhdError):
        x = torch.zeros(4, dtype=torch.float64, device="cuda")
        grmhd.load()
        grmhd._check(grmhd.load().grmhd_arith(5, x.data_ptr(), x.data_ptr(), 4, None), "grmhd_arith")


@pytest.mark.parametrize("fn,c", [("div_sigma", 400.0), ("div_temp", 100.0)])
def test_bound_quotients_bitwise_ieee(dev, fn, c):
    """The bounds' quotients b^2/400 and u/100 by one correction step from
    the divisor's correctly rounded reciprocal: the IEEE quotient bit for bit
    (numpy's division on the host; torch's division of a CUDA tensor by a
    scalar multiplies by the scalar's reciprocal, which is not the IEEE
    quotient), over 1e6 values spread log-uniformly over 1e-290 .. 1e290 and
    powers of two, their multiples of the divisor and the neighbours of
    both."""
    torch, grmhd = dev
    rng = np.random.default_rng(7)
    xs = 10.0 ** rng.uniform(-290.0, 290.0, 1_000_000)
    p2 = 2.0 ** np.arange(-960, 960, 7, dtype=np.float64)
    edge = np.concatenate([p2, np.nextafter(p2, 0.0), np.nextafter(p2, np.inf), p2 * c,
                           np.nextafter(p2 * c, 0.0), np.nextafter(p2 * c, np.inf)])
    xs = np.concatenate([xs, edge])
    a, _ = _run(dev, fn, xs)
    ref = xs / c
    assert np.array_equal(a.view(np.int64), ref.view(np.int64)), int((a != ref).sum())
