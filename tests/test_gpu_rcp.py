"""The reciprocal the step uses inside its arithmetic (WENO5 weights, signal
speeds, the Newton iteration of the 1D_W inversion): the hardware
approximation refined by one third-order step.  Against the IEEE quotient
1/x computed on the same device, it must be within 2 ulp over the normal
range it is specified for, on values spread log-uniformly over 1e-300 ..
1e300 of both signs, on the magnitudes the WENO5 pair feeds it (products
of two sums of squared smoothness indicators) and on exact powers of two.
Outside [2^-1022, 2^1022] the approximation flushes (zero or subnormal
x -> NaN, |x| > 2^1022 -> 0), as the header states."""
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


def test_rcp_within_2_ulp_of_ieee_division(dev):
    torch, grmhd = dev
    rng = np.random.default_rng(7)
    n = 1 << 20
    mag = 10.0 ** rng.uniform(-300, 300, n)
    sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    pows = 2.0 ** np.arange(-1022, 1023, dtype=np.float64)
    xs = np.concatenate([mag * sign, _weno_denominators(rng, n // 4), pows, -pows,
                         np.nextafter(pows, 0.0)[1:], 1.0 + np.arange(1, 4096) * 2.0 ** -52])
    xs = xs[np.isfinite(xs) & (np.abs(xs) >= 2.0 ** -1022) & (np.abs(xs) <= 2.0 ** 1022)]
    x = torch.from_numpy(xs).cuda()
    out = torch.empty_like(x)
    grmhd.rcp(x, out)
    ref = torch.reciprocal(x)  # IEEE division on the device
    torch.cuda.synchronize()
    a, b = out.cpu().numpy(), ref.cpu().numpy()
    assert np.all(np.sign(a) == np.sign(b))
    u = _ulps(a, b)
    assert u.max() <= 2, (int(u.max()), float(xs[int(np.argmax(u))]))
    # and most are exact: the third-order step leaves ~2^-60 before rounding
    assert (u == 0).mean() > 0.9


def test_rcp_outside_the_normal_range(dev):
    """The approximation flushes subnormal inputs and results to zero: a
    zero or subnormal x gives NaN (the refinement meets inf * 0), |x| above
    2^1022 (a subnormal quotient) gives a zero of x's sign."""
    torch, grmhd = dev
    xs = np.array([2.0 ** -1074, -2.0 ** -1040, 0.0, 2.0 ** 1022 * 1.5, -(2.0 ** 1023)])
    x = torch.from_numpy(xs).cuda()
    out = torch.empty_like(x)
    grmhd.rcp(x, out)
    torch.cuda.synchronize()
    a = out.cpu().numpy()
    assert np.all(np.isnan(a[:3]))
    assert a[3] == 0.0 and not np.signbit(a[3])
    assert a[4] == 0.0 and np.signbit(a[4])
