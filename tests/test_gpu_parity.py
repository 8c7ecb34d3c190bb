"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerance.  FP64 rounding (1.1e-16) through the step's ~12k operations per
zone-cycle, with condition growth of at most rho/u ~ 1e3 in the energy
recovery, stays far below 1e-12; the measured differences are <= 4e-14.
After one full predictor-corrector step in FP64, for each primitive group -- rho; u;
utilde^1..3; B^1..3 -- the largest zone difference is <= 1e-12 of the
group's scale, and every zone agrees to 1e-9 relative (plus that floor).
The group scale is the group's largest magnitude, except that velocities
are measured in units of c (scale max(max|utilde|, 1)): the update adds flux
differences of O(p) quantities, so a velocity carries an absolute rounding
error of order machine epsilon whatever its own size.

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
import math

import numpy as np
import pytest

import oracle
from paper_2110_10191_gb300 import problems as pb

pytestmark = pytest.mark.gpu

GROUPS = [(0,), (1,), (2, 3, 4), (5, 6, 7)]
TOL_NORM = 1e-12
TOL_ZONE = 1e-9


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


def compare(a, b, tol_norm=TOL_NORM, tol_zone=TOL_ZONE, what=""):
    """Group-scaled and zone-wise comparison of primitive arrays [8,...]."""
    report = {}
    for grp, scale in zip(GROUPS, group_scales(b)):
        for v in grp:
            d = np.abs(a[v] - b[v])
            if scale == 0.0:
                assert d.max() == 0.0, (what, v)
                continue
            report[v] = d.max() / scale
            assert d.max() <= tol_norm * scale, (what, v, d.max() / scale)
            bad = d > tol_zone * np.abs(b[v]) + tol_norm * scale
            assert not bad.any(), (what, v, int(bad.sum()))
    return report


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
    compare(s.get_prims(), o.get_prims(), tol_norm=1e-9, tol_zone=1e-7, what="own geometry")


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
    rep = compare(s.get_prims(), o.get_prims(), what="mode")
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
    compare(Pg, Po, tol_norm=1e-10, tol_zone=1e-6, what="mode period")


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
    compare(s.get_prims(), o.get_prims(), what=str(shape))
    pfo, ffo = o.flags()
    pfg, ffg = s.flags()
    assert np.array_equal(pfg, pfo)
    mism = ffg != ffo
    # a bound decided at a knife edge may flip with rounding; none expected here
    assert mism.sum() <= max(2, ffo.size // 10000), int(mism.sum())
    co = o.counters()
    assert st["inv_failures"] == co["inv_failures"]
    assert abs(st["floor_hits"] - co["floor_hits"]) <= max(2, ffo.size // 10000)
    assert st["t"] == pytest.approx(o.time()[0], rel=1e-14)


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
    compare(s.get_prims(), o.get_prims(), tol_norm=1e-11, what="bondi")
    assert np.array_equal(s.get_prims(True)[:, :, :, :3], o.get_prims(True)[:, :, :, :3])


def test_predictor_parity(grmhd):
    pr = pb.fm_torus(24, 24, 8)
    o, s = _pair(pr, grmhd)
    o.predictor()
    s.predictor()
    compare(s.get_prims(), o.get_prims(), what="predictor")


def test_orszag_tang_parity(grmhd):
    pr = pb.orszag_tang(48, recon=pb.RECON_WENO5)
    o, s = _pair(pr, grmhd)
    o.step(2)
    s.step(2)
    compare(s.get_prims(), o.get_prims(), tol_norm=1e-11, what="OT")


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
    compare(s.get_prims(), o.get_prims(), what="128^3")


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
