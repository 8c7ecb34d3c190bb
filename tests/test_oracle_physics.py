"""Pins of the oracle's pointwise physics against closed forms and invariants.

* P -> U and P -> F in flat space against the special-relativistic closed
  forms (fluid at rest with a field; moving unmagnetised fluid), b^2 against
  B^2/gamma^2 + (B.v)^2.
* In Kerr (MKS): u.u = -1 and b.u = 0 at random points; the conserved
  densities of a fluid at rest in the normal frame in closed form.
* Signal speeds: +-c_ms at rest; relativistic velocity addition for motion
  along the direction; the transverse-motion closed form; the lapse/shift
  form for the normal frame in Kerr.
* 1D_W inversion: P -> U -> P round trips over random states with Lorentz
  factor up to 50 and sigma up to 400 at MKS points, within the conditioning
  of the conserved variables (and 1e-12 on well-conditioned states); the
  closed-form inversion of a fluid at rest.
* Floors: the paper's bounds hold on exit; untouched zones stay bitwise.
"""
import math
import os

import numpy as np
import pytest

import oracle

A, H = 0.9375, 0.3
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EPS = np.finfo(float).eps


def test_flat_rest_with_field():
    gam = 4.0 / 3.0
    P = np.array([0.7, 0.3, 0, 0, 0, 0.2, -0.5, 0.4])
    U = oracle.prim_to_flux(0, 0, 1, [0, .1, .2, .3], gam, P, 0)
    B2 = 0.2 ** 2 + 0.5 ** 2 + 0.4 ** 2
    ref = np.array([0.7, -0.3 - 0.5 * B2, 0, 0, 0, 0.2, -0.5, 0.4])
    assert np.allclose(U, ref, rtol=1e-15, atol=1e-16)
    # flux along x of a static field: momentum flux = total pressure - B_x B_j
    F = oracle.prim_to_flux(0, 0, 1, [0, .1, .2, .3], gam, P, 1)
    p = (gam - 1) * 0.3
    assert F[0] == 0 and F[1] == 0
    assert F[2] == pytest.approx(p + 0.5 * B2 - 0.2 * 0.2, rel=1e-15)
    assert F[3] == pytest.approx(-0.2 * -0.5, rel=1e-15)
    assert F[4] == pytest.approx(-0.2 * 0.4, rel=1e-15)
    assert np.all(F[5:] == 0)


def test_flat_moving_hydro():
    gam = 5.0 / 3.0
    rng = np.random.default_rng(0)
    for _ in range(20):
        rho, u = rng.uniform(0.1, 2), rng.uniform(0.01, 3)
        ut = rng.normal(size=3) * 2
        P = np.array([rho, u, *ut, 0, 0, 0])
        g = math.sqrt(1 + ut @ ut)
        p = (gam - 1) * u
        w = rho + u + p
        U = oracle.prim_to_flux(0, 0, 1, [0, 0, 0, 0], gam, P, 0)
        assert U[0] == pytest.approx(rho * g, rel=1e-14)
        assert U[1] == pytest.approx(-w * g * g + p + rho * g, rel=1e-12, abs=1e-13 * w * g * g)
        assert np.allclose(U[2:5], w * g * ut, rtol=1e-13)
        for d in (1, 2, 3):
            F = oracle.prim_to_flux(0, 0, 1, [0, 0, 0, 0], gam, P, d)
            vd = ut[d - 1]
            assert F[0] == pytest.approx(rho * vd, rel=1e-14)
            assert F[1] == pytest.approx(-w * g * vd + rho * vd, rel=1e-12, abs=1e-13 * w * g * abs(vd))
            mom = w * vd * ut
            mom[d - 1] += p
            assert np.allclose(F[2:5], mom, rtol=1e-13, atol=1e-14 * w * g * g)


def test_flat_bsq_closed_form():
    rng = np.random.default_rng(1)
    for _ in range(20):
        ut = rng.normal(size=3)
        B = rng.normal(size=3)
        P = np.array([1, 1, *ut, *B])
        g = math.sqrt(1 + ut @ ut)
        v = ut / g
        ref = B @ B / g ** 2 + (B @ v) ** 2
        assert oracle.state_at(0, 0, 1, [0, 0, 0, 0], P)["bsq"] == pytest.approx(ref, rel=1e-13)


def _kerr_points(n, seed):
    rng = np.random.default_rng(seed)
    X = np.zeros((n, 4))
    X[:, 1] = np.log(rng.uniform(1.3, 60.0, n))
    X[:, 2] = rng.uniform(0.02, 0.98, n)
    return rng, X


def test_kerr_invariants():
    rng, Xs = _kerr_points(40, 2)
    for X in Xs:
        G = oracle.geom_at(1, A, H, X)
        P = np.array([1.0, 0.5, *rng.normal(size=3), *rng.normal(size=3)])
        st = oracle.state_at(1, A, H, X, P)
        u, b = st["ucon"], st["bcon"]
        g = G["gcov"]
        assert u @ g @ u == pytest.approx(-1.0, abs=1e-12 * (1 + (np.abs(u) @ np.abs(g) @ np.abs(u))))
        assert abs(b @ g @ u) <= 1e-12 * (np.abs(b) @ np.abs(g) @ np.abs(u))
        assert abs(st["bsq"] - b @ g @ b) <= 1e-13 * (np.abs(b) @ np.abs(g) @ np.abs(b))
        # conserved field = primitive field; flux of B^d along d vanishes
        U = oracle.prim_to_flux(1, A, H, X, 4 / 3, P, 0)
        scale = G["gdet"] * np.abs(b).max() * np.abs(u).max()
        assert np.allclose(U[5:], G["gdet"] * P[5:], rtol=0, atol=1e-14 * scale)
        for d in (1, 2, 3):
            F = oracle.prim_to_flux(1, A, H, X, 4 / 3, P, d)
            assert abs(F[4 + d]) <= 1e-14 * G["gdet"] * np.abs(b).max() * np.abs(u).max() * 4


def test_kerr_normal_frame_densities():
    """utilde = 0: u_mu = (-alpha, 0, 0, 0), b^t = 0, b^i = alpha B^i, so
    U_rho = sqrt(-g) rho/alpha and U_E = sqrt(-g)(rho/alpha - rho - u - b^2/2)
    with b^2 = alpha^2 g_ij B^i B^j."""
    rng, Xs = _kerr_points(20, 3)
    for X in Xs:
        G = oracle.geom_at(1, A, H, X)
        B = rng.normal(size=3)
        P = np.array([0.8, 0.05, 0, 0, 0, *B])
        al, gd = G["alpha"], G["gdet"]
        bsq = al * al * (B @ G["gcov"][1:, 1:] @ B)
        U = oracle.prim_to_flux(1, A, H, X, 4 / 3, P, 0)
        assert U[0] == pytest.approx(gd * 0.8 / al, rel=1e-13)
        assert U[1] == pytest.approx(gd * (0.8 / al - 0.8 - 0.05 - 0.5 * bsq), rel=1e-11)


def test_vchar_flat_rest():
    gam = 4.0 / 3.0
    P = np.array([1.0, 2.0, 0, 0, 0, 0.5, 0.3, -0.2])
    for d in (1, 2, 3):
        vmax, vmin = oracle.vchar(0, 0, 1, [0, 0, 0, 0], gam, P, d)
        ef = 1 + gam * 2.0
        bsq = 0.25 + 0.09 + 0.04
        cs2 = gam * (gam - 1) * 2.0 / ef
        va2 = bsq / (bsq + ef)
        cms = math.sqrt(cs2 + va2 - cs2 * va2)
        assert vmax == pytest.approx(cms, rel=1e-14)
        assert vmin == pytest.approx(-cms, rel=1e-14)


def test_vchar_flat_moving_along():
    gam = 5.0 / 3.0
    for v in (0.3, -0.7, 0.95):
        ut = v / math.sqrt(1 - v * v)
        for d in (1, 2, 3):
            P = np.zeros(8)
            P[0], P[1] = 1.0, 0.4
            P[1 + d] = ut
            cs = math.sqrt(gam * (gam - 1) * 0.4 / (1 + gam * 0.4))
            vmax, vmin = oracle.vchar(0, 0, 1, [0, 0, 0, 0], gam, P, d)
            assert vmax == pytest.approx((v + cs) / (1 + v * cs), rel=1e-13)
            assert vmin == pytest.approx((v - cs) / (1 - v * cs), rel=1e-13)


def test_vchar_flat_transverse_motion():
    """Sound speed along x for a flow moving along y with speed v:
    +- cs sqrt((1 - v^2)(1 - v^2 cs^2)) / (1 - v^2 cs^2)."""
    gam = 4.0 / 3.0
    v = 0.6
    P = np.array([1.0, 0.7, 0, v / math.sqrt(1 - v * v), 0, 0, 0, 0])
    cs2 = gam * (gam - 1) * 0.7 / (1 + gam * 0.7)
    ref = math.sqrt(cs2) * math.sqrt((1 - v * v) * (1 - v * v * cs2)) / (1 - v * v * cs2)
    vmax, vmin = oracle.vchar(0, 0, 1, [0, 0, 0, 0], gam, P, 1)
    assert vmax == pytest.approx(ref, rel=1e-13)
    assert vmin == pytest.approx(-ref, rel=1e-13)


def test_vchar_kerr_normal_frame():
    """A fluid at rest in the normal frame: coordinate speeds along d are
    -beta^d +- alpha sqrt(gamma^{dd}) c_ms (lapse alpha, shift beta^d =
    alpha^2 g^{td}, spatial inverse metric gamma^{dd} = g^{dd} + beta^d beta^d/alpha^2)."""
    gam = 4.0 / 3.0
    rng, Xs = _kerr_points(20, 4)
    for X in Xs:
        G = oracle.geom_at(1, A, H, X)
        B = rng.normal(size=3) * 0.3
        P = np.array([1.0, 0.6, 0, 0, 0, *B])
        bsq = oracle.state_at(1, A, H, X, P)["bsq"]
        ef = 1 + gam * 0.6
        cs2 = gam * (gam - 1) * 0.6 / ef
        va2 = bsq / (bsq + ef)
        cms = math.sqrt(cs2 + va2 - cs2 * va2)
        al = G["alpha"]
        for d in (1, 2, 3):
            beta = al * al * G["gcon"][0, d]
            gdd = G["gcon"][d, d] + beta * beta / (al * al)
            vmax, vmin = oracle.vchar(1, A, H, X, gam, P, d)
            s = al * math.sqrt(gdd) * cms
            assert vmax == pytest.approx(-beta + s, rel=1e-11, abs=1e-13 * s)
            assert vmin == pytest.approx(-beta - s, rel=1e-11, abs=1e-13 * s)


def _random_state(rng, X, gam, gmax=50.0, smax=400.0):
    G = oracle.geom_at(1, A, H, X)
    g = G["gcov"]
    rho = 10 ** rng.uniform(-6, 0)
    u = 10 ** rng.uniform(-8, 1)
    glf = 1 + (gmax - 1) * rng.uniform() ** 3
    d = rng.normal(size=3)
    d /= math.sqrt(d @ g[1:, 1:] @ d)
    ut = d * math.sqrt(glf * glf - 1)
    P = np.array([rho, u, *ut, *rng.normal(size=3)])
    b1 = oracle.state_at(1, A, H, X, P)["bsq"]
    sig = 10 ** rng.uniform(-4, math.log10(smax))
    P[5:] *= math.sqrt(sig * rho / b1)
    return P, glf, sig


def test_inversion_round_trip_conditioned():
    """P -> U -> P, guess 30% off.  Error bounds follow from the conditioning
    of the conserved variables: u is known to eps * E/u with E = (rho +
    gamma_ad u + b^2) gamma^2 (it is a small part of the total energy), rho
    and utilde to eps * gamma^2 (1 + sigma) (through 1 - v^2 = 1/gamma^2)."""
    gam = 4.0 / 3.0
    rng, Xs = _kerr_points(2000, 5)
    for X in Xs:
        P, glf, sig = _random_state(rng, X, gam)
        U = oracle.prim_to_flux(1, A, H, X, gam, P, 0)
        Pg = P.copy()
        Pg[0] *= 1.3
        Pg[1] *= 0.7
        Pg[2:5] *= 0.9
        rc, P2 = oracle.cons_to_prim(1, A, H, X, gam, U, Pg)
        assert rc == 0, (X, P)
        bsq = oracle.state_at(1, A, H, X, P)["bsq"]
        E = (P[0] + gam * P[1] + bsq) * glf ** 2
        c_rho = glf ** 2 * (1 + sig)
        assert abs(P2[0] - P[0]) <= 500 * EPS * c_rho * P[0]
        assert abs(P2[1] - P[1]) <= 500 * EPS * E
        assert np.abs(P2[2:5] - P[2:5]).max() <= 500 * EPS * c_rho * np.abs(P[2:5]).max()
        # B^j = b^j u^t - b^t u^j is formed with that cancellation in U_B
        st = oracle.state_at(1, A, H, X, P)
        ub, bb = st["ucon"], st["bcon"]
        cb = np.abs(bb[1:]) * abs(ub[0]) + abs(bb[0]) * np.abs(ub[1:])
        assert np.all(np.abs(P2[5:] - P[5:]) <= 500 * EPS * cb)


def test_inversion_round_trip_well_conditioned():
    """Lorentz factor <= 2, sigma <= 1, u/rho >= 1e-2: every primitive to 1e-12."""
    gam = 4.0 / 3.0
    rng, Xs = _kerr_points(1000, 6)
    worst = 0.0
    for X in Xs:
        P, glf, sig = _random_state(rng, X, gam, gmax=2.0, smax=1.0)
        P[1] = max(P[1], 1e-2 * P[0])
        U = oracle.prim_to_flux(1, A, H, X, gam, P, 0)
        rc, P2 = oracle.cons_to_prim(1, A, H, X, gam, U, P * 1.01)
        assert rc == 0
        rel = np.abs(P2 - P) / np.maximum(np.abs(P), 1e-300)
        rel[2:5] = np.abs(P2[2:5] - P[2:5]) / np.abs(P[2:5]).max()
        worst = max(worst, rel.max())
    assert worst < 1e-12, worst


def test_inversion_flat_closed_form():
    """Flat space, fluid at rest, field B: U = (rho, -u - B^2/2, 0, B) inverts
    to (rho, u, 0, B) exactly up to rounding."""
    gam = 4.0 / 3.0
    B = np.array([0.3, -0.1, 0.2])
    U = np.array([2.0, -0.5 - 0.5 * (B @ B), 0, 0, 0, *B])
    rc, P = oracle.cons_to_prim(0, 0, 1, [0, 0, 0, 0], gam, U, np.array([1.0, 1.0, 0.1, 0, 0, 0, 0, 0]))
    assert rc == 0
    assert np.allclose(P, [2.0, 0.5, 0, 0, 0, *B], rtol=1e-14, atol=1e-15)


def test_inversion_reports_unphysical():
    """Energy below the rest mass and kinetic energy: no physical state."""
    gam = 4.0 / 3.0
    U = np.array([1.0, +0.5, 0.8, 0, 0, 0, 0, 0])  # U_E > 0 at rest frame = negative thermal energy
    rc, P = oracle.cons_to_prim(0, 0, 1, [0, 0, 0, 0], gam, U, np.array([1, 0.1, 0, 0, 0, 0, 0, 0.]))
    assert rc != 0
    rc, P = oracle.cons_to_prim(0, 0, 1, [0, 0, 0, 0], gam, np.array([-1.0, -1, 0, 0, 0, 0, 0, 0]),
                                np.array([1, 0.1, 0, 0, 0, 0, 0, 0.]))
    assert rc == 6


def _golden_floors():
    vals = {}
    with open(os.path.join(GOLDEN, "floors.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_floors_bounds_hold():
    """After the floors every bound of the paper's list holds at once, and
    each bound that acted leaves its variable on the bound: rho and u end at
    the largest of their lower bounds."""
    gv = _golden_floors()
    gam = 4.0 / 3.0
    rng, Xs = _kerr_points(500, 8)
    hits = 0
    for X in Xs:
        P, glf, sig = _random_state(rng, X, gam, gmax=200.0, smax=1e5)
        P[0] *= 10 ** rng.uniform(-8, 0)
        P[1] *= 10 ** rng.uniform(-8, 0)
        fl, P2 = oracle.floors_at(1, A, H, X, gam, P)
        hits += fl != 0
        r = math.exp(X[1])
        k = 1.0 / (r * r * (1 + r / 10.0))
        G = oracle.geom_at(1, A, H, X)
        bsq = oracle.state_at(1, A, H, X, P2)["bsq"]
        lor = math.sqrt(1 + P2[2:5] @ G["gcov"][1:, 1:] @ P2[2:5])
        assert P2[0] >= gv["rho_floor_coef"] * k * (1 - 1e-15)
        assert P2[1] >= gv["u_floor_coef"] * k ** gam * (1 - 1e-15)
        assert bsq / P2[0] <= gv["sigma_max"] * (1 + 1e-12)
        assert (gam - 1) * P2[1] / (0.5 * bsq) >= gv["beta_min"] * (1 - 1e-12) or bsq == 0
        assert P2[1] / P2[0] <= gv["u_over_rho_max"] * (1 + 1e-15)
        assert lor <= gv["gamma_max"] * (1 + 1e-12)
        if fl == 0:
            assert np.array_equal(P2, P)
        if fl & 1:
            assert lor == pytest.approx(gv["gamma_max"], rel=1e-12)
        # each geometric-floor flag names its own bound: set exactly when the
        # variable came in below that floor
        assert bool(fl & oracle.FF_RHO_GEOM) == bool(P[0] < gv["rho_floor_coef"] * k)
        assert bool(fl & oracle.FF_U_GEOM) == bool(P[1] < gv["u_floor_coef"] * k ** gam)
        # the bounds add the least material: u and rho end at the largest of
        # their lower bounds (b^2 depends on neither, only on the capped
        # velocity and the field)
        u_min = max(P[1], gv["u_floor_coef"] * k ** gam, gv["beta_min"] * bsq / (2 * (gam - 1)))
        assert P2[1] == pytest.approx(u_min, rel=1e-12)
        rho_min = max(P[0], gv["rho_floor_coef"] * k, bsq / gv["sigma_max"],
                      P2[1] / gv["u_over_rho_max"])
        assert P2[0] == pytest.approx(rho_min, rel=1e-12)
    assert hits > 100


def test_floors_leave_good_zones_bitwise():
    gam = 4.0 / 3.0
    X = np.array([0, math.log(10.0), 0.5, 0])
    P = np.array([0.5, 0.1, 0.1, 0.0, 0.02, 1e-3, 1e-3, 0])
    fl, P2 = oracle.floors_at(1, A, H, X, gam, P)
    assert fl == 0 and np.array_equal(P, P2)
