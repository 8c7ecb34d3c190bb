"""Pins of the oracle's full step against what the mathematics fixes.

* A uniform flat state stays exactly uniform (fluxes equal on both faces).
* Periodic flat domain: total mass, energy, momentum and field are conserved
  to round-off (the update telescopes).
* Flux-CT keeps the corner-centred divergence of B unchanged to round-off
  (Toth 2000; paper, "Implementation Notes", first paragraph).
* Linear fast / Alfven / slow modes converge at second order (the paper's
  linear-mode convergence test, "Tests" section).
* The Fishbone-Moncrief torus is a stationary solution: the residual
  S - div F in its interior falls at second order with resolution (source
  terms, connection and fluxes in curved space).
* Equatorial reflection symmetry of the torus is preserved.
* Restart from a checkpoint is bitwise identical to an uninterrupted run
  (the paper's restart identity test, "Tests" section).
* The time step on a uniform state has the closed form of the CFL rule.
* A 3D periodic flat domain conserves everything across all three seams.
* The predictor-corrector is second order in time on a non-stationary
  flow in curved space (the stage state of the geometric source enters).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2110_10191_gb300 import problems as pb

NG = 3


def _uniform_problem(n=(8, 8, 4), P0=None, recon=pb.RECON_WENO5):
    if P0 is None:
        P0 = np.array([1.3, 0.7, 0.2, -0.1, 0.3, 0.4, 0.2, -0.3])
    P = np.empty((8,) + tuple(n[::-1]))
    for v in range(8):
        P[v] = P0[v]
    return pb.Problem(name="uniform", n=n, xmin=(0, 0, 0), xmax=(1, 1, 1), metric=0, a=0.0,
                      hslope=1.0, gamma=5 / 3, cfl=0.8, t_final=0.0, recon=recon, floors=0,
                      bc=((0, 0),) * 3, P=P)


@pytest.mark.parametrize("recon", [pb.RECON_MC, pb.RECON_WENO5])
def test_uniform_state_is_stationary(recon):
    pr = _uniform_problem(recon=recon)
    o = oracle.Oracle(pr)
    o.set_prims(pr.P)
    o.step(3)
    P = o.get_prims()
    # only rounding of the P -> U -> P round trip may differ
    assert np.allclose(P, pr.P, rtol=2e-15, atol=1e-16)
    assert np.array_equal(o.flags()[0], np.zeros_like(o.flags()[0]))


def test_uniform_dt_closed_form():
    P0 = np.array([1.0, 2.0, 0, 0, 0, 0.5, 0.3, -0.2])
    pr = _uniform_problem(n=(16, 8, 4), P0=P0)
    pr.cfl = 0.9
    o = oracle.Oracle(pr)
    o.set_prims(pr.P)
    gam = pr.gamma
    ef = 1 + gam * 2.0
    bsq = 0.25 + 0.09 + 0.04
    cs2 = gam * (gam - 1) * 2.0 / ef
    va2 = bsq / (bsq + ef)
    c = math.sqrt(cs2 + va2 - cs2 * va2)
    dx = [1 / 16, 1 / 8, 1 / 4]
    ref = 1.0 / sum(c / (0.9 * d) for d in dx)
    assert o.next_dt() == pytest.approx(ref, rel=1e-14)


def _zone_U(pr, P):
    """Conserved densities of every interior zone (pointwise oracle call)."""
    n1, n2, n3 = pr.n
    dx = [(pr.xmax[d] - pr.xmin[d]) / pr.n[d] for d in range(3)]
    U = np.zeros_like(P)
    for k in range(n3):
        for j in range(n2):
            for i in range(n1):
                X = [0, pr.xmin[0] + (i + .5) * dx[0], pr.xmin[1] + (j + .5) * dx[1],
                     pr.xmin[2] + (k + .5) * dx[2]]
                U[:, k, j, i] = oracle.prim_to_flux(pr.metric, pr.a, pr.hslope, X, pr.gamma,
                                                    P[:, k, j, i], 0)
    return U


def test_conservation_periodic_flat():
    pr = pb.orszag_tang(24, recon=pb.RECON_WENO5)
    o = oracle.Oracle(pr)
    o.set_prims(pr.P)
    U0 = _zone_U(pr, pr.P).sum(axis=(1, 2, 3))
    o.step(5)
    assert o.counters()["inv_failures"] == 0
    U1 = _zone_U(pr, o.get_prims()).sum(axis=(1, 2, 3))
    scale = np.abs(_zone_U(pr, pr.P)).sum(axis=(1, 2, 3)) + 1.0
    assert np.all(np.abs(U1 - U0) <= 1e-13 * scale), (U1 - U0) / scale


def test_conservation_periodic_flat_3d():
    """The same in three dimensions, with the state varying along every
    axis, so that each periodic seam carries flux."""
    n = (12, 10, 8)
    x = [(np.arange(m) + 0.5) / m for m in n]
    Z, Y, X = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    P0 = np.array([1.0, 0.6, 0.1, -0.05, 0.08, 0.3, 0.2, -0.1])
    P = np.empty((8,) + n[::-1])
    for v in range(8):
        ph = 0.7 * v
        P[v] = P0[v] + 0.05 * (np.sin(2 * math.pi * X + ph) + np.cos(2 * math.pi * Y - ph)
                               + np.sin(2 * math.pi * Z + 2 * ph))
    pr = _uniform_problem(n=n, P0=P0)
    pr.P = P
    o = oracle.Oracle(pr)
    o.set_prims(P)
    U0 = _zone_U(pr, P).sum(axis=(1, 2, 3))
    o.step(3)
    assert o.counters()["inv_failures"] == 0
    P1 = o.get_prims()
    assert not np.allclose(P1, P, rtol=1e-6, atol=0)
    U1 = _zone_U(pr, P1).sum(axis=(1, 2, 3))
    scale = np.abs(_zone_U(pr, P)).sum(axis=(1, 2, 3)) + 1.0
    assert np.all(np.abs(U1 - U0) <= 1e-13 * scale), (U1 - U0) / scale


def corner_divb(pr, Pg):
    """Corner-centred divergence of sqrt(-g) B^i at the interior corners,
    from primitives with ghosts [8][s3][s2][s1]; geometry by the pointwise
    oracle call at zone centres (X3-independent metrics)."""
    s3, s2, s1 = Pg.shape[1:]
    dx = [(pr.xmax[d] - pr.xmin[d]) / pr.n[d] for d in range(3)]
    gd = np.zeros((s2, s1))
    for j in range(s2):
        for i in range(s1):
            X = [0, pr.xmin[0] + (i - NG + .5) * dx[0], pr.xmin[1] + (j - NG + .5) * dx[1], 0]
            gd[j, i] = oracle.geom_at(pr.metric, pr.a, pr.hslope, X)["gdet"]
    GB = Pg[5:8] * gd[None, None]
    n1, n2, n3 = pr.n
    sl = lambda a, b, c: (slice(NG + c, NG + n3 + c), slice(NG + b, NG + n2 + b), slice(NG + a, NG + n1 + a))
    # corner (i,j,k) at the low corner of zone (i,j,k); zones (i-1..i, j-1..j, k-1..k)
    def box_sum(comp, off_d, d):
        tot = 0.0
        for a in (0, -1):
            for b in (0, -1):
                o3 = [a, b]
                o3.insert(d, off_d)
                tot = tot + GB[comp][sl(*o3)]
        return tot
    div = 0.0
    for d in range(3):
        if pr.n[d] == 1:
            continue
        div = div + (box_sum(d, 0, d) - box_sum(d, -1, d)) / (4 * dx[d])
    return div, np.abs(GB).max() / min(dx[d] for d in range(3) if pr.n[d] > 1)


def test_fluxct_preserves_divb_flat():
    pr = pb.orszag_tang(32, recon=pb.RECON_MC)
    # add a divergent part so that the invariant is a non-zero field
    x = (np.arange(32) + 0.5) / 32
    pr.P[5, 0] += 0.1 * np.sin(2 * np.pi * x)[None, :]
    o = oracle.Oracle(pr)
    o.set_prims(pr.P)
    d0, scale = corner_divb(pr, o.get_prims(True))
    o.step(4)
    d1, _ = corner_divb(pr, o.get_prims(True))
    # the discrete divergence of the sampled field is not zero, but it does not change
    assert np.abs(d0).max() > 1e-3 * scale
    assert np.abs(d1 - d0).max() <= 1e-13 * scale


def test_fluxct_preserves_divb_torus():
    pr = pb.fm_torus(24, 24, 8, recon=pb.RECON_WENO5)
    o = oracle.Oracle(pr)
    o.set_prims(pr.P)
    d0, scale = corner_divb(pr, o.get_prims(True))
    o.step(2)
    d1, _ = corner_divb(pr, o.get_prims(True))
    # B from a corner vector potential: divergence-free to round-off, and it stays so
    # (the outermost corners touch the boundary ghosts and are excluded)
    inner = (slice(1, -1), slice(1, -1), slice(1, -1))
    assert np.abs(d0[inner]).max() <= 1e-12 * scale
    assert np.abs(d1[inner]).max() <= 1e-12 * scale


def _mode_error(kind, n):
    pr = pb.linear_mode(n, kind=kind)
    o = oracle.Oracle(pr)
    o.set_prims(pr.P)
    o.step(100000)
    t = o.time()[0]
    assert t == pytest.approx(pr.t_final, rel=1e-14)
    return np.abs(o.get_prims() - pr.exact(t)).mean(axis=(1, 2, 3)).sum()


@pytest.mark.parametrize("kind", ["fast", "alfven", "slow"])
def test_linear_mode_second_order(kind):
    e = [_mode_error(kind, n) for n in (16, 32, 64)]
    orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert orders[-1] > 1.8, (e, orders)
    assert orders[0] > 1.5, (e, orders)
    # the error is a small fraction of the amplitude at 64^2
    assert e[-1] < 0.05 * 1e-4 * 8


def _torus_residual(n):
    pr = pb.fm_torus(n, n, 1, pert=0.0, field=False, recon=pb.RECON_MC)
    o = oracle.Oracle(pr)
    o.set_prims(pr.P)
    F, _ = o.fluxes()
    Pg = o.get_prims(True)
    dx = [(pr.xmax[d] - pr.xmin[d]) / pr.n[d] for d in range(3)]
    res, ref = [], []
    P = pr.P
    for j in range(n):
        for i in range(n):
            if P[0, 0, j, i] < 0.5:
                continue
            I, J, K = i + NG, j + NG, NG
            X = [0, pr.xmin[0] + (i + .5) * dx[0], (j + .5) * dx[1], 0]
            S = oracle.source_at(1, pr.a, pr.hslope, X, pr.gamma, Pg[:, K, J, I])
            div = sum((F[d, :, K + o3[2], J + o3[1], I + o3[0]] - F[d, :, K, J, I]) / dx[d]
                      for d, o3 in enumerate([(1, 0, 0), (0, 1, 0), (0, 0, 1)]))
            res.append(np.abs(S - div)[[0, 1, 2, 3, 4]])
            ref.append(np.abs(S)[[2, 3]].max())
    return np.mean(res, axis=0), np.mean(ref)


def test_torus_equilibrium_residual_second_order():
    r32, s32 = _torus_residual(32)
    r64, s64 = _torus_residual(64)
    # radial and polar momentum residuals shrink ~4x per doubling
    ratio = r32[2:4] / r64[2:4]
    assert np.all(ratio > 3.0), (r32, r64)
    assert r64[2] < 0.05 * s64


def test_torus_equatorial_symmetry():
    pr = pb.fm_torus(24, 24, 4, pert=0.0, recon=pb.RECON_WENO5)
    o = oracle.Oracle(pr)
    o.set_prims(pr.P)
    o.step(3)
    P = o.get_prims()
    M = P[:, :, ::-1, :]
    parity = np.array([1, 1, 1, -1, 1, -1, 1, -1])  # rho u ut1 ut2 ut3 B1 B2 B3
    for v in range(8):
        scale = np.abs(P[v]).max() + 1e-300
        assert np.abs(P[v] - parity[v] * M[v]).max() <= 1e-9 * scale, v


def test_restart_bitwise():
    pr = pb.fm_torus(16, 16, 4, recon=pb.RECON_WENO5)
    a = oracle.Oracle(pr)
    a.set_prims(pr.P)
    a.step(2)
    b = oracle.Oracle(pr)
    b.set_prims(pr.P)
    b.step(1)
    t, dt, ns = b.time()
    ck = b.get_prims(True)
    c = oracle.Oracle(pr)
    c.set_prims(ck)
    c.set_time(t, dt, ns)
    c.step(1)
    assert np.array_equal(a.get_prims(True), c.get_prims(True))
    assert a.time() == c.time()


def test_polar_faces_carry_no_flux():
    pr = pb.fm_torus(16, 16, 4)
    o = oracle.Oracle(pr)
    o.set_prims(pr.P)
    F, _ = o.fluxes()
    n2 = pr.n[1]
    assert np.all(F[1, :, NG:-NG, NG, NG:-NG] == 0.0)
    assert np.all(F[1, :, NG:-NG, NG + n2, NG:-NG] == 0.0)


def test_torus_step_respects_floors():
    gv = {}
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "floors.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                gv[k] = float(v)
    pr = pb.fm_torus(16, 16, 4, recon=pb.RECON_WENO5)
    o = oracle.Oracle(pr)
    o.set_prims(pr.P)
    o.step(2)
    P = o.get_prims()
    dx1 = (pr.xmax[0] - pr.xmin[0]) / 16
    for k in range(4):
        for j in range(16):
            for i in range(16):
                X = [0, pr.xmin[0] + (i + .5) * dx1, (j + .5) / 16, 0]
                r = math.exp(X[1])
                kk = 1 / (r * r * (1 + r / 10))
                p = P[:, k, j, i]
                bsq = oracle.state_at(1, pr.a, pr.hslope, X, p)["bsq"]
                assert p[0] >= gv["rho_floor_coef"] * kk * (1 - 1e-15)
                assert p[1] >= gv["u_floor_coef"] * kk ** pr.gamma * (1 - 1e-15)
                assert bsq <= gv["sigma_max"] * p[0] * (1 + 1e-12)
                assert p[1] <= gv["u_over_rho_max"] * p[0] * (1 + 1e-15)


def _bondi_drift(n):
    pr = pb.bondi(n, n, t_final=5.0, r_in=1.5)
    o = oracle.Oracle(pr)
    o.set_prims(pr.info["P_ghost"])
    assert o.step(100000) == 0
    assert o.counters()["inv_failures"] == 0
    P = o.get_prims()
    return np.abs(P[0] - pr.P[0]).mean() / np.abs(pr.P[0]).mean()


def test_bondi_stationary_second_order():
    """Stationary Michel inflow on Schwarzschild (the paper's Bondi
    convergence test, "Tests" section): the L1 drift of rho after t = 5
    falls at second order, on a fixed domain (r_in = 1.5 inside the
    horizon, R_out = 20, X1 ghosts held at the analytic solution)."""
    e = np.array([_bondi_drift(n) for n in (16, 32, 64)])
    orders = np.log2(e[:-1] / e[1:])
    assert np.all(orders > 1.7), (e, orders)
    assert e[-1] < 1e-4


def _bondi_perturbed(cfl, n=16, t_final=2.0):
    """Michel inflow with a smooth 10% bump in rho and u: a flow in curved
    space that is not stationary, run to t_final on one grid."""
    pr = pb.bondi(n, n, t_final=t_final, r_in=1.5, recon=pb.RECON_WENO5, cfl=cfl)
    Pg = pr.info["P_ghost"].copy()
    s3, s2, s1 = Pg.shape[1:]
    X1, X2 = np.meshgrid((np.arange(s1) - NG + 0.5) / n, (np.arange(s2) - NG + 0.5) / n)
    bump = np.exp(-((X1 - 0.5) ** 2 + (X2 - 0.5) ** 2) / 0.02)
    Pg[0] *= (1 + 0.1 * bump)[None]
    Pg[1] *= (1 + 0.1 * bump)[None]
    o = oracle.Oracle(pr)
    o.set_prims(Pg)
    assert o.step(100000) == 0
    assert o.time()[0] == t_final
    return o.get_prims()


def test_time_integration_second_order_in_curved_space():
    """The predictor-corrector is second order in time: on one grid, the
    difference between runs at CFL 0.4 and 0.2 is 4x that between 0.2 and
    0.1.  The flow is non-stationary and the metric curved, so the
    geometric source's stage state enters (flat or stationary tests cannot
    see it)."""
    P4, P2, P1 = (_bondi_perturbed(c) for c in (0.4, 0.2, 0.1))
    e1 = np.abs(P4 - P2).mean(axis=(1, 2, 3))[:4]
    e2 = np.abs(P2 - P1).mean(axis=(1, 2, 3))[:4]
    assert np.all(e1 / e2 > 3.3), (e1, e2)
