"""Pins of the oracle's drift-frame bounds (the variant of the paper's bounds
list in which floor material is added as a field-free parcel moving with the
drift velocity, the part of the fluid 3-velocity perpendicular to B).

What fixes the variant independently of its own formula:

* Without a field (or one below 1e-20 of the density, whose direction is
  rounding), and for flow perpendicular to the field, the parcel moves
  with the fluid and ideal-MHD stress-energy is linear in (rho, u) at fixed
  4-velocity and field, so the result is the fluid-frame one.
* For flow along the field the drift velocity vanishes: the conserved
  variables gain exactly those of a parcel at rest in the normal frame.
* In general the conserved variables gain those of a field-free parcel of the
  fluid-frame deficits (mass, internal energy) whose 3-velocity v_p is
  perpendicular to B and differs from the fluid's v by a multiple of B,
  which together define the perpendicular projection of v.
* Every bound holds on exit; zones that need no mass or energy are treated
  exactly as in the fluid frame.
"""
import math
import os

import numpy as np
import pytest

import oracle

A, H = 0.9375, 0.3
GAM = 4.0 / 3.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _points(n, seed):
    rng = np.random.default_rng(seed)
    X = np.zeros((n, 4))
    X[:, 1] = np.log(rng.uniform(1.5, 60.0, n))
    X[:, 2] = rng.uniform(0.05, 0.95, n)
    return rng, X


def _floor_k(X):
    r = math.exp(X[1])
    return 1.0 / (r * r * (1 + r / 10.0))


def _state(rng, X, field="random", glf_max=10.0):
    """A state with rho and u below their geometric floors (so a parcel is
    added) and a Lorentz factor below the cap."""
    G = oracle.geom_at(1, A, H, X)
    g = G["gcov"][1:, 1:]
    k = _floor_k(X)
    rho = 1e-6 * k * 10 ** rng.uniform(-3, -0.3)
    u = 1e-8 * k ** GAM * 10 ** rng.uniform(-3, -0.3)
    glf = 1 + (glf_max - 1) * rng.uniform() ** 2
    d = rng.normal(size=3)
    d /= math.sqrt(d @ g @ d)
    ut = d * math.sqrt(glf * glf - 1)
    B = rng.normal(size=3)
    if field == "none":
        B[:] = 0.0
    elif field == "perp":
        ut = ut - (ut @ g @ B) / (B @ g @ B) * B
    elif field == "par":
        B = ut * (rng.uniform(0.5, 2.0) / math.sqrt(ut @ g @ ut))
    # keep b^2 small against the floors so the sigma and beta bounds stay out
    P = np.array([rho, u, *ut, *B])
    if field != "none":
        bsq = oracle.state_at(1, A, H, X, P)["bsq"]
        P[5:] *= math.sqrt((1e-25 if field == "weak" else 1e-3) * rho / bsq)
    return P, G


def _rel(a, b, scale):
    return np.max(np.abs(a - b)) / scale


@pytest.mark.parametrize("field", ["none", "perp", "weak"])
def test_drift_equals_fluid_frame(field):
    """No field, flow perpendicular to the field, and a field too weak to
    have a direction (B^2 below 1e-20 rho, the stated reading): the parcel
    moves with the fluid."""
    rng, Xs = _points(300, {"none": 11, "perp": 12, "weak": 16}[field])
    for X in Xs:
        P, G = _state(rng, X, field)
        fl_f, Pf = oracle.floors_at(1, A, H, X, GAM, P)
        fl_d, Pd, pre = oracle.floors_drift_at(1, A, H, X, GAM, P)
        assert fl_d & oracle.FF_DRIFT and not fl_d & oracle.FF_DRIFT_FAIL
        assert (fl_d & fl_f) == fl_f
        assert Pd[0] == pytest.approx(Pf[0], rel=1e-12)
        assert Pd[1] == pytest.approx(Pf[1], rel=1e-12)
        un = math.sqrt(Pf[2:5] @ G["gcov"][1:, 1:] @ Pf[2:5])
        assert _rel(Pd[2:5], Pf[2:5], max(un, 1e-300)) <= 1e-11
        # B comes back from U_B = sqrt(-g)(b^j u^t - b^t u^j): rounding of |b||u|
        assert _rel(Pd[5:], P[5:], np.abs(P[5:]).max() + 1e-300) <= 1e-13 or np.array_equal(Pd[5:], P[5:])


def test_drift_parallel_flow_adds_a_parcel_at_rest():
    """Flow along B: the drift velocity is zero, so U(P) gains U of (drho,
    du) at rest in the normal frame, utilde = 0."""
    rng, Xs = _points(300, 13)
    for X in Xs:
        P, G = _state(rng, X, "par")
        fl_f, Pf = oracle.floors_at(1, A, H, X, GAM, P)
        fl_d, Pd, pre = oracle.floors_drift_at(1, A, H, X, GAM, P)
        assert fl_d & oracle.FF_DRIFT
        parcel = np.array([Pf[0] - P[0], Pf[1] - P[1], 0, 0, 0, 0, 0, 0])
        dU = oracle.prim_to_flux(1, A, H, X, GAM, pre, 0) - oracle.prim_to_flux(1, A, H, X, GAM, P, 0)
        Up = oracle.prim_to_flux(1, A, H, X, GAM, parcel, 0)
        scale = np.abs(oracle.prim_to_flux(1, A, H, X, GAM, pre, 0)[:5]).max()
        assert _rel(dU[:5], Up[:5], scale) <= 1e-11
        # the parcel slows the parallel flow: momentum is shared with mass at rest
        g = G["gcov"][1:, 1:]
        assert pre[2:5] @ g @ pre[2:5] < P[2:5] @ g @ P[2:5]


def test_drift_parcel_moves_perpendicular_to_the_field():
    """General flow: U(P_pre) - U(P) is the conserved vector of a field-free
    parcel with the fluid-frame deficits whose velocity is the fluid's minus
    a multiple of B and is perpendicular to B."""
    rng, Xs = _points(400, 14)
    checked = 0
    for X in Xs:
        P, G = _state(rng, X, "random")
        g = G["gcov"][1:, 1:]
        fl_f, Pf = oracle.floors_at(1, A, H, X, GAM, P)
        fl_d, Pd, pre = oracle.floors_drift_at(1, A, H, X, GAM, P)
        assert fl_d & oracle.FF_DRIFT
        dU = oracle.prim_to_flux(1, A, H, X, GAM, pre, 0) - oracle.prim_to_flux(1, A, H, X, GAM, P, 0)
        dU[5:] = 0.0
        guess = np.array([Pf[0] - P[0], Pf[1] - P[1], *P[2:5], 0, 0, 0])
        rc, Pp = oracle.cons_to_prim(1, A, H, X, GAM, dU, guess)
        assert rc == 0
        assert Pp[0] == pytest.approx(Pf[0] - P[0], rel=1e-8)
        assert Pp[1] == pytest.approx(Pf[1] - P[1], rel=1e-7)
        v = P[2:5] / math.sqrt(1 + P[2:5] @ g @ P[2:5])
        vp = Pp[2:5] / math.sqrt(1 + Pp[2:5] @ g @ Pp[2:5])
        B = P[5:]
        bn = math.sqrt(B @ g @ B)
        vn = math.sqrt(v @ g @ v)
        assert abs(vp @ g @ B) <= 1e-7 * vn * bn
        lam = ((v - vp) @ g @ B) / (B @ g @ B)
        r = v - vp - lam * B
        assert math.sqrt(abs(r @ g @ r)) <= 1e-7 * vn
        checked += 1
    assert checked == 400


def _golden():
    vals = {}
    with open(os.path.join(GOLDEN, "floors.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_drift_bounds_hold():
    """Every bound of the paper's list holds on exit, as in the fluid frame;
    zones that need only the Lorentz-factor cap, or nothing, come out
    bitwise as in the fluid frame."""
    gv = _golden()
    rng = np.random.default_rng(15)
    X = np.zeros(4)
    hits = same = 0
    for _ in range(600):
        X[1] = math.log(rng.uniform(1.5, 60.0))
        X[2] = rng.uniform(0.02, 0.98)
        G = oracle.geom_at(1, A, H, X)
        g = G["gcov"][1:, 1:]
        rho = 10 ** rng.uniform(-9, 0)
        u = 10 ** rng.uniform(-11, 1)
        glf = 1 + 199 * rng.uniform() ** 3
        d = rng.normal(size=3)
        d /= math.sqrt(d @ g @ d)
        P = np.array([rho, u, *(d * math.sqrt(glf * glf - 1)), *rng.normal(size=3)])
        bsq = oracle.state_at(1, A, H, X, P)["bsq"]
        P[5:] *= math.sqrt(10 ** rng.uniform(-4, 5) * rho / bsq)
        fl_f, Pf = oracle.floors_at(1, A, H, X, GAM, P)
        fl, P2 = oracle.floors_drift_at(1, A, H, X, GAM, P)[:2]
        k = _floor_k(X)
        bsq2 = oracle.state_at(1, A, H, X, P2)["bsq"]
        lor = math.sqrt(1 + P2[2:5] @ g @ P2[2:5])
        assert P2[0] >= gv["rho_floor_coef"] * k * (1 - 1e-15)
        assert P2[1] >= gv["u_floor_coef"] * k ** GAM * (1 - 1e-15)
        assert bsq2 / P2[0] <= gv["sigma_max"] * (1 + 1e-12)
        assert (GAM - 1) * P2[1] / (0.5 * bsq2) >= gv["beta_min"] * (1 - 1e-12) or bsq2 == 0
        assert P2[1] / P2[0] <= gv["u_over_rho_max"] * (1 + 1e-15)
        assert lor <= gv["gamma_max"] * (1 + 1e-12)
        if not fl_f & ~oracle.FF_GAMMA:
            assert fl == fl_f and np.array_equal(P2, Pf)
            same += 1
        else:
            hits += 1
            assert fl & (oracle.FF_DRIFT | oracle.FF_DRIFT_FAIL)
    assert hits > 200 and same > 20
