"""Mixed-precision mode (FP32 reconstruction, fluid states, signal speeds
and LLF fluxes; FP64 geometry, flux-CT, update, 1D_W inversion, bounds):
its error against the FP64 oracle, div B at round-off, second-order
convergence of the linear mode.  The same fluxes with the float-float
update (GRMHD_PREC_MIXED_FF): the same error bound against the oracle, and
within the float-float update's rounding of the mixed mode itself."""
import numpy as np
import pytest

import oracle
from paper_2110_10191_gb300 import problems as pb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def grmhd():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2110_10191_gb300 import grmhd as g
    g.load()
    return g


def _scales(b):
    sc = [max(np.abs(b[v]).max() for v in grp) for grp in ((0,), (1,), (2, 3, 4), (5, 6, 7))]
    sc[2] = max(sc[2], 1.0)
    return [sc[0], sc[1], sc[2], sc[2], sc[2], sc[3], sc[3], sc[3]]


def corner_divb(P, gdet, dx, n):
    """max |corner-centred div(sqrt(-g) B)| over interior corners."""
    GB = P[5:8] * gdet[None, None]
    ng = 3
    def box(comp, off, d):
        tot = 0.0
        for a in (0, -1):
            for b in (0, -1):
                o3 = [a, b]
                o3.insert(d, off)
                tot = tot + GB[comp][ng + o3[2]: ng + n[2] + o3[2], ng + o3[1]: ng + n[1] + o3[1],
                                     ng + o3[0]: ng + n[0] + o3[0]]
        return tot
    div = 0.0
    for d in range(3):
        if n[d] > 1:
            div = div + (box(d, 0, d) - box(d, -1, d)) / (4 * dx[d])
    return np.abs(div[1:-1, 1:-1, 1:-1]).max(), np.abs(GB).max() / min(dx[d] for d in range(3) if n[d] > 1)


def test_mixed_one_step_error_vs_fp64_oracle(grmhd):
    pr = pb.fm_torus(32, 32, 16)
    o = oracle.Oracle(pr)
    o.set_prims(pr.P)
    o.step(1)
    pm = pb.fm_torus(32, 32, 16)
    pm.precision = 1
    s = grmhd.Sim(pm)
    for loc in range(4):
        s.set_geom(loc, o.geom(loc))
    s.set_prims(pm.P)
    s.step(1)
    a, b = s.get_prims(), o.get_prims()
    sc = _scales(b)
    err = [np.abs(a[v] - b[v]).max() / sc[v] for v in range(8)]
    # FP32 fluxes: errors of order the FP32 epsilon, far below the scheme's truncation
    assert max(err) < 1e-5, err
    assert max(err) > 1e-12  # it is genuinely the FP32 path


def test_mixed_divb_round_off(grmhd):
    pr = pb.fm_torus(24, 24, 8)
    pr.precision = 1
    s = grmhd.Sim(pr)
    s.set_prims(pr.P)
    gdet = s.geom(0)[32]
    dx = [(pr.xmax[d] - pr.xmin[d]) / pr.n[d] for d in range(3)]
    d0, scale = corner_divb(s.get_prims(True), gdet, dx, pr.n)
    s.step(5)
    d1, _ = corner_divb(s.get_prims(True), gdet, dx, pr.n)
    assert d0 <= 1e-12 * scale and d1 <= 1e-12 * scale


def test_mixed_linear_mode_converges(grmhd):
    errs = []
    for n in (32, 64, 128):
        pr = pb.linear_mode(n)
        pr.precision = 1
        s = grmhd.Sim(pr)
        s.set_prims(pr.P)
        s.step(100000)
        errs.append(np.abs(s.get_prims() - pr.exact(pr.t_final)).mean(axis=(1, 2, 3)).sum())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[0] > 1.7, (errs, orders)


def test_mixed_orszag_tang_close_to_fp64(grmhd):
    pr = pb.orszag_tang(64, recon=pb.RECON_WENO5)
    s64 = grmhd.Sim(pr)
    s64.set_prims(pr.P)
    s64.step(10)
    pm = pb.orszag_tang(64, recon=pb.RECON_WENO5)
    pm.precision = 1
    sm = grmhd.Sim(pm)
    sm.set_prims(pm.P)
    sm.step(10)
    a, b = sm.get_prims(), s64.get_prims()
    sc = _scales(b)
    assert max(np.abs(a[v] - b[v]).max() / sc[v] for v in range(8)) < 1e-4


def test_mixed_ff_one_step_error_vs_fp64_oracle(grmhd):
    """Mixed fluxes with the float-float update: the FP32 fluxes still set
    the error, and the result is the mixed mode's up to the update's
    rounding (the float-float bar, 3e-11 of each group's scale)."""
    pr = pb.fm_torus(32, 32, 16)
    o = oracle.Oracle(pr)
    o.set_prims(pr.P)
    o.step(1)
    out = {}
    for prec in (1, 3):
        pm = pb.fm_torus(32, 32, 16)
        pm.precision = prec
        s = grmhd.Sim(pm)
        for loc in range(4):
            s.set_geom(loc, o.geom(loc))
        s.set_prims(pm.P)
        s.step(1)
        out[prec] = s.get_prims()
    b = o.get_prims()
    sc = _scales(b)
    err = [np.abs(out[3][v] - b[v]).max() / sc[v] for v in range(8)]
    assert max(err) < 1e-5, err
    diff = [np.abs(out[3][v] - out[1][v]).max() / sc[v] for v in range(8)]
    assert max(diff) < 3e-11, diff
    assert max(diff) > 0  # it is genuinely the float-float update


def test_mixed_ff_divb_and_orszag_tang(grmhd):
    pr = pb.fm_torus(24, 24, 8)
    pr.precision = 3
    s = grmhd.Sim(pr)
    s.set_prims(pr.P)
    gdet = s.geom(0)[32]
    dx = [(pr.xmax[d] - pr.xmin[d]) / pr.n[d] for d in range(3)]
    s.step(5)
    d1, scale = corner_divb(s.get_prims(True), gdet, dx, pr.n)
    assert d1 <= 1e-12 * scale
    po = pb.orszag_tang(64, recon=pb.RECON_WENO5)
    s64 = grmhd.Sim(po)
    s64.set_prims(po.P)
    s64.step(10)
    po.precision = 3
    sm = grmhd.Sim(po)
    sm.set_prims(po.P)
    sm.step(10)
    a, b = sm.get_prims(), s64.get_prims()
    sc = _scales(b)
    assert max(np.abs(a[v] - b[v]).max() / sc[v] for v in range(8)) < 1e-4


def test_torus_288_all_modes_vs_oracle(grmhd):
    """The largest workload, the 288x128x128 torus reaching R_out = 1000,
    one step of every precision mode against one FP64 oracle step on the
    same geometry: FP64 within 1e-12 of each group's scale (and 1e-9 per
    zone), float-float within 3e-11, the two FP32-flux modes within 1e-5;
    div B at round-off in all four."""
    def problem(prec):
        pr = pb.fm_torus(288, 128, 128, recon=pb.RECON_WENO5, r_out=1000.0)
        pr.precision = prec
        return pr

    pr = problem(0)
    o = oracle.Oracle(pr)
    o.set_prims(pr.P)
    o.step(1)
    b = o.get_prims()
    sc = _scales(b)
    geom = [o.geom(loc) for loc in range(4)]
    gdet = geom[0][32]
    dx = [(pr.xmax[d] - pr.xmin[d]) / pr.n[d] for d in range(3)]
    bars = {0: 1e-12, 2: 3e-11, 1: 1e-5, 3: 1e-5}
    for prec, bar in bars.items():
        pm = problem(prec)
        s = grmhd.Sim(pm)
        for loc in range(4):
            s.set_geom(loc, geom[loc])
        s.set_prims(pm.P)
        s.step(1)
        a = s.get_prims()
        err = [np.abs(a[v] - b[v]).max() / sc[v] for v in range(8)]
        assert max(err) <= bar, (prec, err)
        if prec == 0:
            for v in range(8):
                bad = np.abs(a[v] - b[v]) > 1e-9 * np.abs(b[v]) + 1e-12 * sc[v]
                assert not bad.any(), (v, int(bad.sum()))
        d, scale = corner_divb(s.get_prims(True), gdet, dx, pm.n)
        assert d <= 1e-12 * scale, (prec, d / scale)
        s.close()
