"""The float-float mode (GRMHD_PREC_FF): reconstruction, fluid states,
signal speeds and LLF fluxes in pairs of FP32 words (about 48 significant
bits) on the FP32 pipe, everything else FP64.

Tolerance.  The FP64 mode's bar scaled by the unit roundoff: a float pair
rounds at 2^-48 (3.6e-15) where FP64 rounds at 2^-53, 32 times finer, so the
one-step bar of 1e-12 of each primitive group's scale becomes 3e-11 (and
1e-9 zone-wise as before).  Fluxes themselves meet the FP64 flux bar
(1e-12).  Measured after one step: 1.5e-14 to 6.6e-14 on the mode, the
vortex and the WENO5 torus; 1.1e-11 on the MC torus, in floor-density
atmosphere zones beside the torus edge, where the update divides rounding
of the edge fluxes by a density near the floor (the FP64 mode shows the
same amplification at 2.5e-14)."""
import numpy as np
import pytest

import oracle
from paper_2110_10191_gb300 import problems as pb
from test_gpu_parity import GROUPS, compare, compare_fluxes, field_scale, group_scales

pytestmark = pytest.mark.gpu

FF = 2
TOL_FF = 3e-11


@pytest.fixture(scope="module")
def grmhd():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2110_10191_gb300 import grmhd as g
    g.load()
    return g


def _pair(pr, grmhd):
    o = oracle.Oracle(pr)
    Pg = pr.info.get("P_ghost") if pr.info else None
    P0 = Pg if Pg is not None else pr.P
    o.set_prims(P0)
    pf = pb.Problem(**{**pr.__dict__})
    pf.precision = FF
    s = grmhd.Sim(pf)
    for loc in range(4):
        s.set_geom(loc, o.geom(loc))
    s.set_prims(P0)
    return o, s


@pytest.mark.parametrize("shape,recon", [((24, 20, 8), pb.RECON_WENO5), ((24, 20, 8), pb.RECON_MC),
                                         ((13, 11, 7), pb.RECON_WENO5), ((32, 32, 1), pb.RECON_WENO5)])
def test_ff_step_parity_torus(grmhd, shape, recon):
    pr = pb.fm_torus(*shape, recon=recon)
    o, s = _pair(pr, grmhd)
    o.step(1)
    s.step(1)
    compare(s.get_prims(), o.get_prims(), tol=TOL_FF, what="ff %s" % (shape,), rule="group")
    pfo, _ = o.flags()
    pfg, _ = s.flags()
    assert np.array_equal(pfg, pfo)


@pytest.mark.parametrize("prob", ["mode", "ot", "bondi"])
def test_ff_step_parity_flat(grmhd, prob):
    if prob == "mode":
        pr, n = pb.linear_mode(64), 1
    elif prob == "ot":
        pr, n = pb.orszag_tang(48, recon=pb.RECON_WENO5), 2
    else:
        pr, n = pb.bondi(32, 24, n3=2, recon=pb.RECON_WENO5), 3
    o, s = _pair(pr, grmhd)
    o.step(n)
    s.step(n)
    compare(s.get_prims(), o.get_prims(), tol=TOL_FF, what="ff " + prob, rule="group")


@pytest.mark.parametrize("recon", [pb.RECON_MC, pb.RECON_WENO5])
def test_ff_flux_parity(grmhd, recon):
    pr = pb.fm_torus(24, 20, 6, recon=recon)
    o, s = _pair(pr, grmhd)
    Fo, co = o.fluxes()
    Fg, cg = s.fluxes()
    assert np.allclose(cg, co, rtol=1e-12, atol=0)
    compare_fluxes(Fg, Fo, field_scale(o, pr))


def test_ff_multi_step_drift(grmhd):
    pr = pb.fm_torus(24, 24, 8)
    o, s = _pair(pr, grmhd)
    o.step(5)
    s.step(5)
    a, b = s.get_prims(), o.get_prims()
    for grp, sc in zip(GROUPS, group_scales(b)):
        for v in grp:
            assert np.abs(a[v] - b[v]).max() <= 1e-10 * sc, v


def test_ff_in_batch_bitwise(grmhd):
    """Float-float grids share batches with FP64 and mixed grids and give
    their alone results bitwise."""
    probs = pb.batch_2d(ngrid=4, nmin=12, nmax=32, seed=13) + [pb.fm_torus(20, 16, 4)]
    for q, pr in enumerate(probs):
        pr.precision = q % 3
    ref = []
    for pr in probs:
        s = grmhd.Sim(pr)
        s.set_prims(pr.P)
        s.step(2, sync=False)
        ref.append(s.get_prims(with_ghosts=True))
        s.close()
    sims = []
    for pr in probs:
        s = grmhd.Sim(pr)
        s.set_prims(pr.P)
        sims.append(s)
    b = grmhd.Batch(sims)
    b.step(2, sync=True)
    for s, P, pr in zip(sims, ref, probs):
        assert np.array_equal(s.get_prims(with_ghosts=True), P), (pr.name, pr.precision)
    b.close()


def test_ff_flat_equals_full_extent(grmhd):
    pr = pb.orszag_tang(24, recon=pb.RECON_WENO5)
    pr.precision = FF
    ext = pb.Problem(**{**pr.__dict__})
    ext.n = (pr.n[0], pr.n[1], 2)
    ext.xmax = (pr.xmax[0], pr.xmax[1], 1.0e300)
    ext.P = np.concatenate([pr.P, pr.P], axis=1)
    out = []
    for p in (pr, ext):
        s = grmhd.Sim(p)
        s.set_prims(p.P)
        s.step(2)
        out.append(s.get_prims(with_ghosts=True))
        s.close()
    for k in range(2):
        assert np.array_equal(out[1][:, 3 + k, 3:-3, 3:-3], out[0][:, 3, 3:-3, 3:-3]), k


def test_ff_full_size_torus_vs_fp64(grmhd):
    """The bench's 128^3 torus: one float-float step against the FP64 step
    (itself held to the oracle at 1e-12)."""
    pr = pb.fm_torus(128, 128, 128)
    out = []
    for prec in (0, FF):
        p = pb.Problem(**{**pr.__dict__})
        p.precision = prec
        s = grmhd.Sim(p)
        s.set_prims(pr.P)
        s.step(1)
        out.append(s.get_prims())
        s.close()
    compare(out[1], out[0], tol=TOL_FF, what="ff 128^3", rule="group")
