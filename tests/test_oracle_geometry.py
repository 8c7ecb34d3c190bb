"""Pins of the oracle's geometry against facts the mathematics fixes.

* g_{mu nu} g^{nu lambda} = delta (inverse).
* sqrt(-g) of Kerr in MKS has the closed form Sigma |sin theta| r dtheta/dX2.
* Kerr is a vacuum solution: the Ricci tensor built from the oracle's
  numerical connection (finite differences of it) vanishes.  Any typo in a
  metric component, in the MKS Jacobian or an index slip in the connection
  formula breaks this.
* Minkowski: connection identically zero.
The paper fixes the approach (metric quantities evaluated numerically from
the analytic line element): "Implementation Notes", second paragraph.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2110_10191_gb300 import problems as pb

A, H = 0.9375, 0.3


def _points(n=12, seed=1):
    rng = np.random.default_rng(seed)
    X = np.zeros((n, 4))
    X[:, 1] = np.log(rng.uniform(1.3, 60.0, n))
    X[:, 2] = rng.uniform(0.03, 0.97, n)
    X[:, 3] = rng.uniform(0, 2 * math.pi, n)
    return X


def test_inverse_metric():
    for X in _points():
        G = oracle.geom_at(1, A, H, X)
        prod = G["gcov"] @ G["gcon"]
        assert np.max(np.abs(prod - np.eye(4))) < 1e-13 * max(1.0, np.abs(G["gcov"]).max())


def test_gdet_closed_form():
    for X in _points():
        G = oracle.geom_at(1, A, H, X)
        r = math.exp(X[1])
        th = math.pi * X[2] + 0.5 * (1 - H) * math.sin(2 * math.pi * X[2])
        sig = r * r + A * A * math.cos(th) ** 2
        ref = sig * abs(math.sin(th)) * r * math.pi * (1 + (1 - H) * math.cos(2 * math.pi * X[2]))
        assert G["gdet"] == pytest.approx(ref, rel=1e-13)
        assert G["alpha"] == pytest.approx(1.0 / math.sqrt(-G["gcon"][0, 0]), rel=1e-15)


def test_metric_symmetric_and_lapse():
    for X in _points():
        G = oracle.geom_at(1, A, H, X)
        assert np.array_equal(G["gcov"], G["gcov"].T)
        # Kerr-Schild: g^{tt} = -(1 + 2r/Sigma), independent of the MKS stretch
        r = math.exp(X[1])
        th = math.pi * X[2] + 0.5 * (1 - H) * math.sin(2 * math.pi * X[2])
        sig = r * r + A * A * math.cos(th) ** 2
        assert G["gcon"][0, 0] == pytest.approx(-(1 + 2 * r / sig), rel=1e-12)


def _conn(X):
    return oracle.geom_at(1, A, H, X)["conn"]


def test_kerr_ricci_flat():
    """R_{mu nu} = d_l G^l_{mu nu} - d_nu G^l_{mu l} + G^l_{l s} G^s_{mu nu}
    - G^l_{nu s} G^s_{mu l} = 0 for Kerr (vacuum)."""
    h = 2e-3
    for X in _points(8, seed=7):
        G0 = _conn(X)
        dG = np.zeros((4, 4, 4, 4))  # dG[m] = d_m Gamma
        for m in (1, 2, 3):
            vals = []
            for s in (-2, -1, 1, 2):
                Xs = X.copy()
                Xs[m] += s * h
                vals.append(_conn(Xs))
            dG[m] = (vals[0] - 8 * vals[1] + 8 * vals[2] - vals[3]) / (12 * h)
        R = np.zeros((4, 4))
        scale = np.zeros((4, 4))
        for mu in range(4):
            for nu in range(4):
                t1 = sum(dG[l][l, mu, nu] for l in range(4))
                t2 = sum(dG[nu][l, mu, l] for l in range(4))
                t3 = sum(G0[l, l, s] * G0[s, mu, nu] for l in range(4) for s in range(4))
                t4 = sum(G0[l, nu, s] * G0[s, mu, l] for l in range(4) for s in range(4))
                R[mu, nu] = t1 - t2 + t3 - t4
                scale[mu, nu] = abs(t1) + abs(t2) + abs(t3) + abs(t4)
        assert np.all(np.abs(R) <= 2e-6 * scale.max()), (X, np.abs(R).max(), scale.max())


def test_ricci_pin_detects_wrong_metric():
    """Sanity of the pin itself: Schwarzschild with a wrong g_rr factor is not
    Ricci flat, and the same estimator sees it (evaluated here in numpy)."""
    def gcov(X):
        r, th = X[1], X[2]
        g = np.diag([-(1 - 2 / r), 1.0 / (1 - 2 / r) * 1.01, r * r, (r * math.sin(th)) ** 2])
        return g

    def conn(X, d=1e-5):
        g = gcov(X)
        gi = np.linalg.inv(g)
        dg = np.zeros((4, 4, 4))
        for m in (1, 2):
            Xp, Xm = X.copy(), X.copy()
            Xp[m] += d
            Xm[m] -= d
            dg[m] = (gcov(Xp) - gcov(Xm)) / (2 * d)
        return 0.5 * (np.einsum("lk,mkn->lmn", gi, dg) + np.einsum("lk,nkm->lmn", gi, dg)
                      - np.einsum("lk,kmn->lmn", gi, dg))

    X = np.array([0.0, 7.0, 1.1, 0.0])
    h = 1e-2
    dG = np.zeros((4, 4, 4, 4))
    for m in (1, 2):
        v = []
        for s in (-2, -1, 1, 2):
            Xs = X.copy()
            Xs[m] += s * h
            v.append(conn(Xs))
        dG[m] = (v[0] - 8 * v[1] + 8 * v[2] - v[3]) / (12 * h)
    G0 = conn(X)
    R = (np.einsum("llmn->mn", dG) - np.einsum("nlml->mn", dG)
         + np.einsum("lls,smn->mn", G0, G0) - np.einsum("lns,sml->mn", G0, G0))
    assert np.abs(R).max() > 1e-4


def test_minkowski_connection_zero():
    G = oracle.geom_at(0, 0.0, 1.0, [0, 0.3, 0.6, 0.2])
    assert np.all(G["conn"] == 0.0)
    assert np.array_equal(G["gcov"], np.diag([-1.0, 1, 1, 1]))
    assert G["gdet"] == 1.0 and G["alpha"] == 1.0


def test_geometry_arrays_match_pointwise():
    pr = pb.fm_torus(8, 8, 2, field=False)
    o = oracle.Oracle(pr)
    g = o.geom(0)
    dx1 = (pr.xmax[0] - pr.xmin[0]) / 8
    dx2 = 1.0 / 8
    i, j = 5, 4  # with ghosts
    X = [0, pr.xmin[0] + (i - 3 + 0.5) * dx1, (j - 3 + 0.5) * dx2, 0]
    G = oracle.geom_at(1, pr.a, pr.hslope, X)
    assert g[32, j, i] == G["gdet"]
    assert np.array_equal(g[:16, j, i].reshape(4, 4), G["gcov"])
    gf = o.geom(1)
    Xf = [0, pr.xmin[0] + (i - 3) * dx1, X[2], 0]
    assert gf[32, j, i] == oracle.geom_at(1, pr.a, pr.hslope, Xf)["gdet"]
