"""Pins of the oracle's boundary conditions by what they must continue or
forbid, not by their formulas.

* Polar ghosts (the X2 ends of a Kerr grid, theta = 0 and pi).  Take an
  axisymmetric field that is smooth through the axis. Its X1 and X3
  components are even in theta across the axis, and its X2 component is
  odd (e_theta turns over).  The ghosts past the pole must hold that
  continuation: the field evaluated at the ghost centres.
* Outflow ghosts (the X1 ends).  A monopole field, B^1 = C/sqrt(-g), is
  divergence-free.  The ghosts must continue it divergence-free, i.e. with
  sqrt(-g) B^1 = C.
* An outflow boundary lets nothing in.  Where the gas at the edge moves
  into the grid, the ghosts carry no inward velocity and the mass flux
  through the boundary face is zero.  Where the gas leaves, the flux is
  kept.
"""
import math

import numpy as np

import oracle
from paper_2110_10191_gb300 import problems as pb

NG = oracle.NG


def _centres(pr, d, count):
    """Zone-centre coordinates along d for indices -NG .. n+NG-1."""
    dx = (pr.xmax[d] - pr.xmin[d]) / pr.n[d]
    return pr.xmin[d] + (np.arange(-NG, count + NG) + 0.5) * dx


def test_polar_ghosts_continue_axisymmetric_fields():
    pr = pb.fm_torus(16, 16, 4)
    n1, n2, n3 = pr.n
    x1 = _centres(pr, 0, n1)
    x2 = _centres(pr, 1, n2)
    X1, X2 = np.meshgrid(x1, x2)  # [s2][s1]
    even = 1.0 + 0.3 * np.cos(2 * math.pi * X2)   # even about X2 = 0 and X2 = 1
    odd = np.sin(2 * math.pi * X2)                 # odd about both
    radial = 1.0 + 0.1 * X1
    F = np.array([radial * even, 0.1 * even, 0.01 * even * radial, 0.02 * odd, 0.03 * even,
                  0.1 * even, 0.3 * odd * radial, 0.05 * even])  # [8][s2][s1]
    P = np.ascontiguousarray(np.broadcast_to(F[:, None], (8, n3 + 2 * NG, n2 + 2 * NG, n1 + 2 * NG)))
    o = oracle.Oracle(pr)
    o.set_prims(np.ascontiguousarray(P[:, NG:-NG, NG:-NG, NG:-NG]))
    G = o.get_prims(with_ghosts=True)
    ks, iss = slice(NG, NG + n3), slice(NG, NG + n1)
    for rows in (slice(0, NG), slice(NG + n2, n2 + 2 * NG)):
        got = G[:, ks, rows, iss]
        want = P[:, ks, rows, iss]
        for v in range(8):
            scale = np.abs(F[v]).max()
            assert np.abs(got[v] - want[v]).max() <= 1e-13 * scale, (v, rows)


def test_outflow_ghosts_continue_a_monopole():
    pr = pb.fm_torus(16, 8, 4)
    n1, n2, n3 = pr.n
    o = oracle.Oracle(pr)
    gdet = o.geom(0)[32]  # zone-centre sqrt(-g), [s2][s1]
    C = 0.1
    P = np.zeros((8, n3, n2, n1))
    P[0], P[1] = 1.0, 0.1
    P[5] = (C / gdet[NG:-NG, NG:-NG])[None]
    o.set_prims(P)
    G = o.get_prims(with_ghosts=True)
    js, ks = slice(NG, NG + n2), slice(NG, NG + n3)
    for cols in (slice(0, NG), slice(NG + n1, n1 + 2 * NG)):
        flux = G[5, ks, js, cols] * gdet[None, js, cols]
        assert np.abs(flux - C).max() <= 1e-14 * C, cols
        assert np.all(G[6:8, ks, js, cols] == 0.0)


def test_outflow_boundaries_let_nothing_in():
    """The inner X1 edge lies inside the horizon, where every mass flux
    points into the hole whatever the gas's normal-frame velocity; the
    outer edge is where inflow has to be stopped."""
    pr = pb.fm_torus(16, 8, 4)
    n1, n2, n3 = pr.n
    js, ks = slice(NG, NG + n2), slice(NG, NG + n3)
    o = oracle.Oracle(pr)
    P = pr.P.copy()
    P[2, :, :, :3] = 0.5      # pushing away from the hole at the inner edge
    P[2, :, :, -3:] = -0.05   # moving inwards at the outer edge: into the grid
    o.set_prims(P)
    G = o.get_prims(with_ghosts=True)
    assert np.all(G[2, :, :, :NG] <= 0.0)
    assert np.all(G[2, :, :, NG + n1:] >= 0.0)
    F, _ = o.fluxes()
    assert np.all(F[0, 0, ks, js, NG] <= 0.0)
    assert np.all(F[0, 0, ks, js, NG + n1] >= 0.0)
    # where the gas leaves, it does
    P[2, :, :, -3:] = 0.05
    o.set_prims(P)
    F, _ = o.fluxes()
    assert np.all(F[0, 0, ks, js, NG] < 0.0)
    assert np.all(F[0, 0, ks, js, NG + n1] > 0.0)
