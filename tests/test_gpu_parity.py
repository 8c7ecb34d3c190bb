"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerance.  After one full predictor-corrector step in FP64 every zone is
held to 1e-12 relative, per primitive (compare(), rule "zone"):
  rho  |a - b| <= 1e-12 max(|b|, 1e-12 max|b|);
  u    the same in every zone where that is coarser than the rounding the
       energy variable carries; in cold zones (u < 3.6e-3 rho) |a - b| <=
       32 eps rho: the energy density and its face fluxes are differences
       of O(rho) terms (rest mass), so two FP64 implementations' u differ
       by a few eps rho however small u is (measured: <= 13 eps rho);
  B^i  |a - b| sqrt(g_ii) <= 1e-12 of the field strength sqrt(g_ij B^i
       B^j) over the zone's domain of dependence of one step (zones within
       6): a component is built from EMF differences of the reconstructed
       states around it, so it carries rounding of that field strength even
       where it crosses zero or sits in a field-free zone beside a
       magnetised one;
  utilde^i  |a - b| <= 1e-12 max(max|utilde|, 1) (units of c: the update
       adds flux differences of O(p) quantities, so a velocity carries an
       absolute rounding of order eps whatever its own size).
FP64 rounding (1.1e-16) through the step's ~12k operations per zone-cycle
stays far below these bars: measured <= 4.4e-13 (rho), 3.1e-13 (u, warm
zones), 5.4e-16 (B), 5.3e-15 (utilde).  Reduced-precision modes and
several-step runs use rule "group" (each variable against its group's
largest magnitude).

Both sides take the same decisions (MC/minmod branches, Newton stopping,
bounds, failures) in FP64; the differences are rounding (FMA contraction on
the GPU, operation order).  The numerical connection (centred differences of
step 1e-5) turns a last-bit difference of the metric into a ~1e-11 relative
difference of Gamma, which near the horizon reaches the velocities at
~1e-10.  So the 1e-12 step tests run both sides on the same geometry (the
oracle's, loaded through grmhd_set_geometry), the GPU's own geometry is
compared with the oracle's separately, and a step on the GPU's own geometry
is held to 1e-9.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2110_10191_gb300 import problems as pb

pytestmark = pytest.mark.gpu

GROUPS = [(0,), (1,), (2, 3, 4), (5, 6, 7)]
NAMES = ["rho", "u", "u1", "u2", "u3", "B1", "B2", "B3"]
TOL = 1e-12          # the one-step FP64 bar
ZONE_FLOOR = 1e-12   # denominator floor, as a fraction of the largest magnitude over zones
EPS = 2.0 ** -53     # FP64 unit roundoff
# The energy variable's rest-mass cancellation: each side forms the energy
# density and the six face fluxes of energy (with the Lax-Friedrichs term
# c U) from pairs of O(rho) terms (T^d_t + rho u^d), each rounding to about
# 2 eps rho, so two implementations' u may differ by up to 2 x 8 x 2 eps rho
# whatever u is.
U_REST_MASS = 32 * EPS
# One full step reads the zones within 3 of a zone per stage: its domain of
# dependence is the cube of zones within 6.
REACH = 6


@pytest.fixture(scope="module")
def grmhd():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2110_10191_gb300 import grmhd as g
    g.load()
    return g


def group_scales(b):
    sc = [max(np.abs(b[v]).max() for v in grp) for grp in GROUPS]
    sc[2] = max(sc[2], 1.0)  # velocities in units of c
    return sc


def zone_rel(a, b):
    """|a - b| / max(|b|, 1e-12 max|b|) per zone (zero where both vanish)."""
    m = np.abs(b).max()
    if m == 0.0:
        return np.where(a == b, 0.0, np.inf)
    return np.abs(a - b) / np.maximum(np.abs(b), ZONE_FLOOR * m)


def _report(what, rep):
    """With GRMHD_PARITY_REPORT set to a path, append the measured figures of
    one comparison as a JSON line (before any assertion), so that a run
    records every comparison's figures, passing or not."""
    path = os.environ.get("GRMHD_PARITY_REPORT")
    if not path:
        return
    rec = {"test": os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0], "what": what}
    rec.update(rep)
    with open(path, "a") as f:
        f.write(json.dumps(rec) + "\n")


def _spatial_metric(ref, shape):
    """g_ij (i, j = 1..3) at the interior zone centres, broadcast to the
    primitive shape [n3, n2, n1]; the identity without a reference."""
    g = np.zeros((3, 3) + tuple(shape))
    if ref is None:
        for i in range(3):
            g[i, i] = 1.0
        return g
    gc = ref.geom(0)[:16, 3:-3, 3:-3]
    for i in range(3):
        for j in range(3):
            g[i, j] = gc[4 * (i + 1) + (j + 1)][None]
    return g


def _reach_max(x):
    """The largest value of x over each zone's domain of dependence of one
    step (the zones within REACH along every axis, clipped at the grid)."""
    from scipy.ndimage import maximum_filter
    return maximum_filter(x, size=2 * REACH + 1, mode="nearest")


def compare(a, b, tol=TOL, what="", ref=None, rule="zone"):
    """Primitive arrays a (CUDA path) against b (oracle), [8, n3, n2, n1].

    rule="zone", the one-step FP64 bar, zone by zone:
      rho:   |a - b| / max(|b|, 1e-12 max|b|) <= tol;
      u:     the same, except in cold zones, where it is finer than the
             rest-mass cancellation of the energy variable allows (32 eps
             rho > 1e-12 u): there |a - b| <= 32 eps rho (U_REST_MASS),
             scaled by tol / 1e-12;
      B^i:   |a - b| sqrt(g_ii) <= tol max(|B|_reach, 1e-12 max|B|), with
             |B| = sqrt(g_ij B^i B^j) the field strength and |B|_reach its
             largest value over the zone's domain of dependence of one step:
             the induction update forms each component from EMF differences
             of b^i u^j - b^j u^i of reconstructed states, so a component
             carries rounding of the field strength around it, whatever its
             own size (it may cross zero, or sit in a field-free zone beside
             a magnetised one);
      utilde^i: |a - b| <= tol max(max|utilde|, 1) (units of c: the update
             adds flux differences of O(p) quantities, so a velocity carries
             an absolute rounding of order eps whatever its own size).
    ref (the oracle holding b): its centre metric for |B| (identity without
    it) and its last stage's bound flags, which split the figures into
    bound-held zones and the others.  rule="group" (reduced precision,
    several steps): every variable to tol times its group's largest
    magnitude.  Returns {variable: largest measured figure}."""
    shape = b.shape[1:]
    held = None if ref is None else (ref.flags()[1] != 0)
    scales = group_scales(b)
    figs, classes, worst, extra = {}, {}, {}, {}
    bad = []
    if rule == "zone":
        g = _spatial_metric(ref, shape)
        Bv = b[5:8]
        bmag = np.sqrt(np.maximum(np.einsum("i...,ij...,j...->...", Bv, g, Bv), 0.0))
        bden = np.maximum(_reach_max(bmag), ZONE_FLOOR * bmag.max()) if bmag.max() > 0 else None
        cold = U_REST_MASS * np.abs(b[0]) > TOL * np.abs(b[1])
        extra["u_cold_zones"] = int(cold.sum())
    for q, grp in enumerate(GROUPS):
        for v in grp:
            d = np.abs(a[v] - b[v])
            if rule == "zone" and v == 0:
                r = zone_rel(a[v], b[v])
            elif rule == "zone" and v == 1:
                r = zone_rel(a[v], b[v])
                extra["u_hot_max"] = float(r[~cold].max()) if (~cold).any() else 0.0
                if cold.any():
                    rc = d / (U_REST_MASS * (tol / TOL) * np.maximum(np.abs(b[0]), 1e-300)) * tol
                    extra["u_cold_max_over_eps_rho"] = float((d / (EPS * np.abs(b[0])))[cold].max())
                    extra["u_cold_max_rel"] = float(r[cold].max())
                    r = np.where(cold, rc, r)
            elif rule == "zone" and v >= 5:
                if bden is None:
                    r = np.where(a[v] == b[v], 0.0, np.inf)
                else:
                    r = d * np.sqrt(g[v - 5, v - 5]) / bden
                    # the same against the zone's own field strength, for the record
                    own = d * np.sqrt(g[v - 5, v - 5]) / np.maximum(bmag, ZONE_FLOOR * bmag.max())
                    extra["%s_vs_own_field" % NAMES[v]] = float(own.max())
            else:
                r = d / scales[q] if scales[q] > 0 else np.where(a[v] == b[v], 0.0, np.inf)
            figs[NAMES[v]] = float(r.max())
            if held is not None:
                classes[NAMES[v]] = {"bound_held": float(r[held].max()) if held.any() else 0.0,
                                     "free": float(r[~held].max()) if (~held).any() else 0.0}
            if r.max() > 0:
                iz = np.unravel_index(int(np.argmax(r)), r.shape)
                worst[NAMES[v]] = {"zone": [int(x) for x in iz], "b": float(b[v][iz]),
                                   "rho": float(b[0][iz]), "u": float(b[1][iz])}
            if not r.max() <= tol:
                bad.append((NAMES[v], figs[NAMES[v]], int((r > tol).sum())))
    _report(what, {"rule": rule, "tol": tol, "max": figs, "classes": classes, "worst": worst,
                   "extra": extra})
    assert not bad, (what, rule, tol, bad)
    return figs


def compare_fluxes(Fg, Fo, Ub_scale, tol=1e-12):
    """Per direction: hydrodynamic fluxes against the largest hydrodynamic
    flux magnitude (they are all built from T^d_nu terms of that size); the
    induction fluxes against the conserved field times c (they are b^j u^d -
    b^d u^j plus the Lax-Friedrichs term c_top (U_B,R - U_B,L), so a weak flux
    in a strong field carries rounding of the field's size)."""
    for d in range(3):
        for grp in ((0, 1, 2, 3, 4), (5, 6, 7)):
            sc = max(np.abs(Fo[d, v]).max() for v in grp)
            if grp[0] == 5:
                sc = max(sc, Ub_scale)
            for v in grp:
                diff = np.abs(Fg[d, v] - Fo[d, v]).max()
                assert diff <= tol * max(sc, 1e-300), (d, v, diff / max(sc, 1e-300))


def field_scale(o, problem):
    """max over zones of sqrt(-g) |B| (the conserved field)."""
    gd = o.geom(0)[32][3:-3, 3:-3]
    return float((np.abs(problem.P[5:8]).max(axis=0).max(axis=0) * gd).max())


def _pair(problem, grmhd, same_geometry=True):
    o = oracle.Oracle(problem)
    o.set_prims(problem.P)
    s = grmhd.Sim(problem)
    if same_geometry:
        for loc in range(4):
            s.set_geom(loc, o.geom(loc))
    s.set_prims(problem.P)
    return o, s


def test_geometry_parity_torus(grmhd):
    """The GPU's own geometry against the oracle's: metric components to 1e-13
    of sqrt(R_m R_n) at each point (R_m the largest component of row m),
    sqrt(-g) and the lapse to 1e-13, the
    connection to 1e-9 of the largest Gamma^l of the point (finite
    differences amplify last-bit metric differences by 1/delta = 1e5)."""
    # the bench's radial grid (128 zones, 5.5 inside the horizon); a grid of
    # 20 radial zones puts its ghost zones near the ring singularity, where the
    # 4x4 inverse is ill-conditioned
    pr = pb.fm_torus(128, 64, 1)
    o, s = _pair(pr, grmhd, same_geometry=False)
    for loc in (0, 1, 2):
        go, gg = o.geom(loc), s.geom(loc)
        for blk in (0, 16):
            # scale of row m: its largest component (diagonal entries such as
            # g_tt at the ergosphere or g^11 at the horizon cross zero)
            rows = [np.max([np.abs(go[blk + 4 * m + n]) for n in range(4)], axis=0) for m in range(4)]
            for m in range(4):
                for n in range(4):
                    c = blk + 4 * m + n
                    sc = np.sqrt(rows[m] * rows[n])
                    assert np.all(np.abs(gg[c] - go[c]) <= 1e-13 * sc + 1e-300), (loc, c)
        for c in (32, 33):
            assert np.all(np.abs(gg[c] - go[c]) <= 1e-13 * np.abs(go[c])), (loc, c)
    co, cg = o.geom(3), s.geom(3)
    for l in range(4):
        blk = slice(16 * l, 16 * l + 16)
        sc = np.abs(co[blk]).max(axis=0)
        assert np.all(np.abs(cg[blk] - co[blk]) <= 1e-9 * sc + 1e-300), l


def test_step_parity_own_geometry(grmhd):
    """One step of the torus on the GPU's own geometry: geometry-limited
    agreement (1e-9)."""
    pr = pb.fm_torus(24, 24, 8)
    o, s = _pair(pr, grmhd, same_geometry=False)
    o.step(1)
    s.step(1)
    compare(s.get_prims(), o.get_prims(), tol=1e-9, what="own geometry", ref=o)


def test_ghost_fill_parity(grmhd):
    for pr in (pb.fm_torus(16, 12, 5), pb.linear_mode(12, n2=9)):
        o, s = _pair(pr, grmhd)
        assert np.array_equal(o.get_prims(True), s.get_prims(True)), pr.name


@pytest.mark.parametrize("recon", [pb.RECON_MC, pb.RECON_WENO5])
def test_flux_parity_torus(grmhd, recon):
    pr = pb.fm_torus(24, 20, 6, recon=recon)
    o, s = _pair(pr, grmhd)
    Fo, co = o.fluxes()
    Fg, cg = s.fluxes()
    assert np.allclose(cg, co, rtol=1e-13, atol=0)
    compare_fluxes(Fg, Fo, field_scale(o, pr))
    assert s.next_dt() == pytest.approx(o.next_dt(), rel=1e-13)


def test_flux_parity_flat_mode(grmhd):
    pr = pb.linear_mode(64)
    o, s = _pair(pr, grmhd)
    Fo, co = o.fluxes()
    Fg, cg = s.fluxes()
    compare_fluxes(Fg, Fo, field_scale(o, pr))


def test_step_parity_linear_mode(grmhd):
    """Linear fast mode, 64 x 64, MC (the accuracy workload): one step."""
    pr = pb.linear_mode(64)
    o, s = _pair(pr, grmhd)
    o.step(1)
    s.step(1)
    rep = compare(s.get_prims(), o.get_prims(), what="mode", ref=o)
    assert s.stats()["t"] == pytest.approx(o.time()[0], rel=1e-14)


def test_linear_mode_full_period(grmhd):
    """One period of the fast mode: the GPU reaches t_final exactly and its
    error against the analytic eigenmode equals the oracle's."""
    pr = pb.linear_mode(64)
    o, s = _pair(pr, grmhd)
    o.step(100000)
    st = s.step(100000)
    assert st["t"] == pytest.approx(pr.t_final, rel=1e-14)
    Pg, Po = s.get_prims(), o.get_prims()
    ex = pr.exact(pr.t_final)
    eg = np.abs(Pg - ex).mean(axis=(1, 2, 3)).sum()
    eo = np.abs(Po - ex).mean(axis=(1, 2, 3)).sum()
    assert eg == pytest.approx(eo, rel=1e-6)
    compare(Pg, Po, tol=1e-10, what="mode period", rule="group")


@pytest.mark.parametrize("shape,recon", [((32, 32, 16), pb.RECON_WENO5),
                                         ((24, 20, 8), pb.RECON_MC),
                                         ((13, 11, 7), pb.RECON_WENO5),
                                         ((32, 32, 1), pb.RECON_WENO5)])
def test_step_parity_torus(grmhd, shape, recon):
    """Kerr torus (MKS, WENO5/MC), ragged sizes and the 2D axisymmetric form:
    one step, primitives, failure codes and bound flags."""
    pr = pb.fm_torus(*shape, recon=recon)
    o, s = _pair(pr, grmhd)
    o.step(1)
    st = s.step(1)
    pfo, ffo = o.flags()
    compare(s.get_prims(), o.get_prims(), what=str(shape), ref=o)
    pfg, ffg = s.flags()
    assert np.array_equal(pfg, pfo)
    mism = ffg != ffo
    # a bound decided at a knife edge may flip with rounding; none expected here
    assert mism.sum() <= max(2, ffo.size // 10000), int(mism.sum())
    co = o.counters()
    assert st["inv_failures"] == co["inv_failures"]
    assert abs(st["floor_hits"] - co["floor_hits"]) <= max(2, ffo.size // 10000)
    assert st["t"] == pytest.approx(o.time()[0], rel=1e-14)


def test_step_parity_unmagnetised_torus(grmhd):
    """B = 0, the degenerate case of the field terms: the magnetosonic speed
    is the sound speed (b^2 = 0), 1D_W has no field (B^2 = Q.B = 0), flux-CT
    carries zero EMFs.  Two steps, primitives and flags against the oracle;
    the field stays exactly zero."""
    pr = pb.fm_torus(24, 20, 8, field=False)
    o, s = _pair(pr, grmhd)
    o.step(2)
    s.step(2)
    Pg, Po = s.get_prims(), o.get_prims()
    compare(Pg, Po, what="B = 0", ref=o)
    assert not Pg[5:8].any() and not Po[5:8].any()
    assert np.array_equal(s.flags()[0], o.flags()[0])


@pytest.mark.parametrize("shape,rw", [((37, 21, 9), 16), ((24, 20, 8), 4), ((32, 32, 1), 2)])
def test_step_parity_walk_lengths(grmhd, shape, rw):
    """The reconstruction's column walk (forced on grids the automatic choice
    gives one thread per zone) against the oracle: two steps."""
    pr = pb.fm_torus(*shape)
    o, s = _pair(pr, grmhd)
    assert s.set_recon_walk(rw) == rw
    o.step(2)
    s.step(2)
    compare(s.get_prims(), o.get_prims(), what="walk %d %s" % (rw, shape), ref=o)
    assert np.array_equal(s.flags()[0], o.flags()[0])


def test_bondi_fixed_boundary_parity(grmhd):
    """Michel inflow with X1 ghosts held at the analytic solution (fixed
    boundaries) and the bounds on: three steps against the oracle."""
    pr = pb.bondi(32, 24, n3=2, recon=pb.RECON_WENO5)
    o = oracle.Oracle(pr)
    o.set_prims(pr.info["P_ghost"])
    s = grmhd.Sim(pr)
    for loc in range(4):
        s.set_geom(loc, o.geom(loc))
    s.set_prims(pr.info["P_ghost"])
    o.step(3)
    s.step(3)
    compare(s.get_prims(), o.get_prims(), tol=1e-11, what="bondi", ref=o)
    assert np.array_equal(s.get_prims(True)[:, :, :, :3], o.get_prims(True)[:, :, :, :3])


def test_predictor_parity(grmhd):
    pr = pb.fm_torus(24, 24, 8)
    o, s = _pair(pr, grmhd)
    o.predictor()
    s.predictor()
    compare(s.get_prims(), o.get_prims(), what="predictor", ref=o)


def test_orszag_tang_parity(grmhd):
    pr = pb.orszag_tang(48, recon=pb.RECON_WENO5)
    o, s = _pair(pr, grmhd)
    o.step(2)
    s.step(2)
    compare(s.get_prims(), o.get_prims(), tol=1e-11, what="OT", ref=o)


def test_multi_step_torus_drift(grmhd):
    """Five steps of the small torus: rounding differences grow but stay small."""
    pr = pb.fm_torus(24, 24, 8)
    o, s = _pair(pr, grmhd)
    o.step(5)
    s.step(5)
    a, b = s.get_prims(), o.get_prims()
    for grp, sc in zip(GROUPS, group_scales(b)):
        for v in grp:
            assert np.abs(a[v] - b[v]).max() <= 1e-10 * sc, v


def test_full_size_torus_one_step(grmhd):
    """The 128^3 WENO5 torus, one step, every zone against the oracle."""
    pr = pb.fm_torus(128, 128, 128)
    o, s = _pair(pr, grmhd)
    o.step(1)
    s.step(1)
    compare(s.get_prims(), o.get_prims(), what="128^3", ref=o)


def test_restart_bitwise_gpu(grmhd):
    pr = pb.fm_torus(16, 16, 8)
    a = grmhd.Sim(pr)
    a.set_prims(pr.P)
    a.step(2)
    b = grmhd.Sim(pr)
    b.set_prims(pr.P)
    st = b.step(1)
    ck = b.get_prims(True)
    c = grmhd.Sim(pr)
    c.set_prims(ck)
    c.set_time(st["t"], st["dt"], st["steps"])
    c.step(1)
    assert np.array_equal(a.get_prims(True), c.get_prims(True))


def test_deterministic_bitwise(grmhd):
    """Two runs of the same state give the same bits (no data races, no
    order dependence in the reductions)."""
    pr = pb.linear_mode(32)
    s1 = grmhd.Sim(pr)
    s1.set_prims(pr.P)
    s1.step(3)
    a = s1.get_prims()
    s2 = grmhd.Sim(pr)
    s2.set_prims(pr.P)
    s2.step(3)
    assert np.array_equal(a, s2.get_prims())


def test_t_final_stops(grmhd):
    pr = pb.linear_mode(16)
    s = grmhd.Sim(pr)
    s.set_prims(pr.P)
    st = s.step(1000)
    P1 = s.get_prims()
    st2 = s.step(3)
    assert st2["t"] == st["t"] == pytest.approx(pr.t_final, rel=1e-14)
    assert np.array_equal(P1, s.get_prims())


def test_device_pointer_io(grmhd):
    import torch
    pr = pb.linear_mode(16)
    s = grmhd.Sim(pr, stream=torch.cuda.current_stream())
    P = torch.from_numpy(pr.P.copy()).cuda()
    s.set_prims(P)
    out = torch.empty_like(P)
    s.get_prims(out=out)
    torch.cuda.synchronize()
    assert torch.equal(out.cpu(), torch.from_numpy(pr.P))


def test_invalid_arguments(grmhd):
    pr = pb.linear_mode(8)
    bad = pb.linear_mode(8)
    bad.recon = 7
    with pytest.raises(grmhd.GrmhdError) as e:
        grmhd.Sim(bad)
    assert e.value.code == -1
    bad = pb.fm_torus(8, 2, 2)  # polar reflection needs n2 >= 3
    with pytest.raises(grmhd.GrmhdError):
        grmhd.Sim(bad)
    s = grmhd.Sim(pr)
    with pytest.raises(ValueError):
        s.set_prims(np.zeros((8, 1, 8, 7)))


def _flat_uniform(n):
    P = np.empty((8,) + tuple(n[::-1]))
    for v, x in enumerate([1.0, 0.5, 0.1, 0.2, 0.0, 0.3, 0.0, 0.1]):
        P[v] = x
    return pb.Problem(name="uniform", n=n, xmin=(0, 0, 0), xmax=(1, 1, 1), metric=0, a=0.0,
                      hslope=1.0, gamma=4 / 3, cfl=0.5, t_final=0.0, recon=pb.RECON_WENO5,
                      floors=0, bc=((0, 0),) * 3, P=P)


def test_unit_grid_has_no_time_step(grmhd):
    """Degenerate 1 x 1 x 1 grid: no direction has a CFL constraint, so there
    is no finite time step; both sides refuse to step."""
    pr = _flat_uniform((1, 1, 1))
    o, s = _pair(pr, grmhd)
    assert o.step(1) == -3
    with pytest.raises(grmhd.GrmhdError) as e:
        s.step(1)
    assert e.value.code == -5
    assert np.array_equal(s.get_prims(), pr.P)


def test_tiny_grid_uniform(grmhd):
    """2 x 1 x 1 periodic grid (narrower than the stencil): stays uniform."""
    pr = _flat_uniform((2, 1, 1))
    o, s = _pair(pr, grmhd)
    o.step(2)
    s.step(2)
    assert np.allclose(s.get_prims(), o.get_prims(), rtol=1e-14, atol=1e-16)
    assert np.allclose(s.get_prims(), pr.P, rtol=1e-14, atol=1e-16)


def test_fp64_peak_probe(grmhd):
    f = grmhd.fp64_peak(1 << 14)
    assert 1e11 < f < 1e14


def test_fp64_issue_rate_probe(grmhd):
    """The FP64 issue rate per SM per clock, with the clock measured in the
    kernel: positive, at most the nominal 2 per SM per clock, and the same
    (within 3%) with one chain per thread as with 8, and with one block per
    SM as with 8."""
    r8, mhz = grmhd.fp64_probe(0, 8, 8, 1 << 12)
    r1, _ = grmhd.fp64_probe(0, 1, 8, 1 << 15)
    rb, _ = grmhd.fp64_probe(0, 8, 1, 1 << 15)
    assert abs(rb / r8 - 1.0) < 0.03
    assert 300.0 < mhz < 4000.0
    assert 0.5 < r8 <= 2.02 and 0.5 < r1 <= 2.02
    assert abs(r1 / r8 - 1.0) < 0.03
    with pytest.raises(grmhd.GrmhdError):
        grmhd.fp64_probe(0, 3, 8, 16)


def _divb_ref(P, gdet, dx, n):
    """Corner-centred divergence of sqrt(-g) B over the corners between
    interior zones, written out with numpy (the definition in grmhd.h)."""
    GB = P[5:8] * gdet[None, None]
    ng = 3
    rng = [(ng + 1, ng + n[d]) if n[d] > 1 else (ng, ng + 1) for d in range(3)]

    def sl(d, o):
        return slice(rng[d][0] + o, rng[d][1] + o)
    div = 0.0
    gb = 0.0
    for d in range(3):
        if n[d] <= 1:
            continue
        tot = 0.0
        for dk in (-1, 0):
            for dj in (-1, 0):
                for di in (-1, 0):
                    v = GB[d][sl(2, dk), sl(1, dj), sl(0, di)]
                    gb = max(gb, np.abs(v).max())
                    tot = tot + (v if (di, dj, dk)[d] == 0 else -v)
        div = div + tot / (4 * dx[d])
    return np.abs(div).max(), gb


def test_divb_diagnostic(grmhd):
    """grmhd_divb against the numpy definition on a field that is not
    divergence-free, and at round-off after CT steps of the torus."""
    pr = pb.fm_torus(20, 16, 6)
    rng = np.random.default_rng(3)
    P = pr.P.copy()
    P[5:8] += 1e-3 * rng.standard_normal(P[5:8].shape)
    s = grmhd.Sim(pr)
    s.set_prims(P)
    gdet = s.geom(0)[32]
    dx = [(pr.xmax[d] - pr.xmin[d]) / pr.n[d] for d in range(3)]
    dg, gg = s.divb()
    dr, gr = _divb_ref(s.get_prims(True), gdet, dx, pr.n)
    assert dg == pytest.approx(dr, rel=1e-12) and gg == pytest.approx(gr, rel=1e-15)
    s2 = grmhd.Sim(pr)
    s2.set_prims(pr.P)
    s2.step(4)
    d4, g4 = s2.divb()
    assert d4 <= 1e-12 * g4 / min(dx)
