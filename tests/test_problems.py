"""Pins of the seeded input generators (set-up arithmetic, not the step).

* Linear-mode eigen-speeds: Alfven speed v_A cos(theta_kB), and for k
  perpendicular to B the fast speed is c_ms; for k along B the sound speed
  c_s and v_A (relativistic closed forms).
* Fishbone-Moncrief torus: log-enthalpy zero at the inner edge, maximum at
  r_max on the equator, unit 4-velocity, max rho = 1 after normalisation.
* Counter-based random numbers depend only on (seed, zone index).
"""
import math

import numpy as np
import pytest

from paper_2110_10191_gb300 import problems as pb


def _speeds(P0, gam, khat):
    lam, _ = pb.mode_eigensystem(np.array(P0, float), gam, np.array(khat, float))
    return np.sort(lam[lam > 1e-10])


def _cs_va(rho, u, bsq, gam):
    ef = rho + gam * u
    cs2 = gam * (gam - 1) * u / ef
    va2 = bsq / (bsq + ef)
    return cs2, va2


def test_alfven_speed_oblique():
    gam = 4 / 3
    s = _speeds([1, 1, 0, 0, 0, 1, 0, 0], gam, [1 / math.sqrt(2), 1 / math.sqrt(2)])
    cs2, va2 = _cs_va(1, 1, 1, gam)
    assert s[1] == pytest.approx(math.sqrt(va2) / math.sqrt(2), rel=1e-10)


def test_fast_speed_perpendicular():
    gam = 4 / 3
    s = _speeds([1, 1, 0, 0, 0, 0, 1.0, 0], gam, [1, 0])
    cs2, va2 = _cs_va(1, 1, 1, gam)
    assert s[-1] == pytest.approx(math.sqrt(cs2 + va2 - cs2 * va2), rel=1e-10)


def test_parallel_speeds():
    gam = 5 / 3
    s = _speeds([1, 0.5, 0, 0, 0, 0.8, 0, 0], gam, [1, 0])
    cs2, va2 = _cs_va(1, 0.5, 0.64, gam)
    got = sorted(set(np.round(s, 12)))
    assert any(abs(x - math.sqrt(cs2)) < 1e-10 for x in got)
    assert any(abs(x - math.sqrt(va2)) < 1e-10 for x in got)


def test_mode_is_real_and_divergence_free():
    pr = pb.linear_mode(16, kind="fast")
    dP = pr.info["dP"]
    k = np.array(pr.info["k"])
    assert abs(dP[5] * k[0] + dP[6] * k[1]) < 1e-12
    assert pr.info["period"] == pytest.approx(1 / (pr.info["speed"] * math.sqrt(2)), rel=1e-14)


def test_fm_torus_enthalpy():
    a, rin, rmax = 0.9375, 6.0, 12.0
    ell = pb.fm_ell(a, rmax)
    assert float(pb.fm_lnh(np.array(rin), np.array(math.pi / 2), a, ell, rin)) == 0.0
    r = np.linspace(8, 20, 24001)
    lnh = pb.fm_lnh(r, np.full_like(r, math.pi / 2), a, ell, rin)
    assert r[np.argmax(lnh)] == pytest.approx(rmax, abs=1e-3)


def test_fm_torus_four_velocity():
    pr = pb.fm_torus(16, 16, 2, field=True)
    P = pr.P
    assert P[0].max() == pytest.approx(1.0, rel=1e-3)
    dx1 = (pr.xmax[0] - pr.xmin[0]) / 16
    X1 = pr.xmin[0] + (np.arange(16) + 0.5) * dx1
    X2 = (np.arange(16) + 0.5) / 16
    X1g, X2g = np.meshgrid(X1, X2, indexing="xy")
    g = pb.mks_gcov(np.exp(X1g), X2g, pr.a, pr.hslope)
    ut = np.stack([P[2, 0], P[3, 0], P[4, 0]], -1)
    gam = np.sqrt(1 + np.einsum("...i,...ij,...j->...", ut, g[..., 1:, 1:], ut))
    assert np.all(gam >= 1.0) and np.all(np.isfinite(gam))
    inside = P[0, 0] > 1e-3
    # in the torus the orbital speed is sub-relativistic but not zero
    assert np.all(gam[inside] < 1.5) and np.any(gam[inside] > 1.01)


def test_splitmix_reproducible():
    idx = np.arange(1000, dtype=np.uint64)
    a = pb.splitmix_uniform(7, idx)
    b = pb.splitmix_uniform(7, idx[::-1])[::-1]
    assert np.array_equal(a, b)
    assert 0.0 <= a.min() and a.max() < 1.0
    assert abs(a.mean() - 0.5) < 0.05
    assert not np.array_equal(a, pb.splitmix_uniform(8, idx))


def test_michel_solution():
    """Michel inflow: constant mass flux 4 pi r^2 rho |u^r| = mdot, the sonic
    point where (u^r)^2 = 1/(2 r_c), temperature rising inward, through the
    horizon."""
    r = np.array([1.2, 1.9, 2.5, 4.0, 8.0, 12.0, 30.0])
    rho, u, ur = pb.michel_state(r, r_c=8.0, mdot=1.0)
    assert np.allclose(4 * math.pi * r * r * rho * np.abs(ur), 1.0, rtol=1e-10)
    assert abs(ur[4]) == pytest.approx(math.sqrt(1 / 16.0), rel=1e-6)
    T = (4 / 3 - 1) * u / rho
    assert np.all(np.diff(T) < 0) and np.all(ur < 0)


def test_batch_2d_recipe():
    """64 grids: N in [32, 256], equal quarters of the four kinds, modes on
    oblique integer wavenumbers with amplitude in [1e-4, 1e-2], vortex scale
    in [0.5, 1.5], deterministic, and grid g independent of the grid count."""
    import collections
    probs = pb.batch_2d()
    assert len(probs) == 64
    kinds = collections.Counter(p.info["kind"] for p in probs)
    assert kinds == {k: 16 for k in pb.BATCH_KINDS}
    for p in probs:
        n1, n2, n3 = p.n
        assert n1 == n2 and n3 == 1 and 32 <= n1 <= 256
        assert p.metric == pb.METRIC_MINKOWSKI and p.bc == ((pb.BC_PERIODIC,) * 2,) * 3
        assert p.P.shape == (8, 1, n1, n1) and np.isfinite(p.P).all()
        if p.info["kind"] == "orszag_tang":
            assert 0.5 <= p.info["scale"] <= 1.5
        else:
            assert 1e-4 <= p.info["amp"] <= 1e-2
            kx, ky = (k / (2 * np.pi) for k in p.info["k"])
            assert (round(kx), round(ky)) in pb.BATCH_WAVENUMBERS
            # the mode is the requested branch: slow < Alfven < fast
            lam = sorted(x for x in p.info["eigenvalues"] if x > 1e-10)
            pos = {"slow": 0, "alfven": 1, "fast": len(lam) - 1}[p.info["kind"]]
            assert p.info["speed"] == pytest.approx(lam[pos])
    again = pb.batch_2d()
    assert all(np.array_equal(a.P, b.P) for a, b in zip(probs, again))
    few = pb.batch_2d(ngrid=8)
    # the kind shares depend on ngrid; sizes, reconstruction and draws do not
    assert [p.n for p in few] == [p.n for p in probs[:8]]
    assert [p.recon for p in few] == [p.recon for p in probs[:8]]


def test_serving_stream_recipe():
    """200 Poisson arrivals at 4/s: 60/40 tori/Bondi, sizes, spins, cycle
    counts and precisions in their ranges, deterministic."""
    st = pb.serving_stream()
    assert len(st) == 200 and st == pb.serving_stream()
    t = np.array([r["t_arrival"] for r in st])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert 0.2 < gaps.mean() < 0.3                      # 1/rate = 0.25 s
    tori = [r for r in st if r["kind"] == "torus"]
    assert 0.5 < len(tori) / 200 < 0.7
    for r in st:
        assert 20 <= r["steps"] <= 200 and r["precision"] in (0, 1)
        if r["kind"] == "torus":
            assert 64 <= r["n"] <= 192 and 0.0 <= r["a"] <= 0.98
        else:
            assert 96 <= r["n"] <= 160
    assert 0.35 < np.mean([r["precision"] for r in st]) < 0.65
    small = pb.serving_problem({"id": 3, "kind": "bondi", "n": 96, "a": 0.0, "steps": 20,
                                "precision": 1, "t_arrival": 0.0})
    assert small.n == (96, 96, 96) and small.precision == 1
