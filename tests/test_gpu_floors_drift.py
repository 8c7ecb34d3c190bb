"""Drift-frame bounds on the GPU (GRMHD_FLOOR_DRIFT) against the oracle's
drift-frame bounds, and their consistency with the rest of the library.

* One step of the Kerr torus (whose atmosphere sits on the floors) with the
  bounds in the drift frame: primitives within the FP64 one-step bar (1e-12
  of each group's scale), failure codes exactly, bound flags but for knife
  edges.  Float-float grids within that mode's bar (3e-11).
* The predictor in both frames: zones that no bound touched are bitwise
  equal, zones with a drift-frame parcel carry the drift flag.
* Batched, decomposed and single grids give bitwise the same evolution.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2110_10191_gb300 import problems as pb

from test_gpu_parity import compare

pytestmark = pytest.mark.gpu

TOL_FF = 3e-11
FF_DRIFT, FF_DRIFT_FAIL = 64, 128


@pytest.fixture(scope="module")
def grmhd():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2110_10191_gb300 import grmhd as g
    g.load()
    return g


def _drift(pr, **kw):
    return dataclasses.replace(pr, floor_frame=1, **kw)


def _pair(pr, grmhd):
    o = oracle.Oracle(pr)
    o.set_prims(pr.P)
    s = grmhd.Sim(pr)
    for loc in range(4):
        s.set_geom(loc, o.geom(loc))
    s.set_prims(pr.P)
    return o, s


@pytest.mark.parametrize("shape,recon", [((32, 32, 16), pb.RECON_WENO5),
                                         ((24, 20, 8), pb.RECON_MC),
                                         ((32, 32, 1), pb.RECON_WENO5)])
def test_drift_step_parity_torus(grmhd, shape, recon):
    pr = _drift(pb.fm_torus(*shape, recon=recon))
    o, s = _pair(pr, grmhd)
    o.step(1)
    st = s.step(1)
    compare(s.get_prims(), o.get_prims(), what="drift %s" % (shape,), ref=o)
    pfo, ffo = o.flags()
    pfg, ffg = s.flags()
    assert np.array_equal(pfg, pfo)
    assert (ffo & FF_DRIFT).sum() > 100  # the atmosphere takes parcels
    mism = ffg != ffo
    assert mism.sum() <= max(2, ffo.size // 10000), int(mism.sum())
    co = o.counters()
    assert st["inv_failures"] == co["inv_failures"]
    assert abs(st["floor_hits"] - co["floor_hits"]) <= max(2, ffo.size // 10000)


def test_drift_step_parity_float_float(grmhd):
    pr = _drift(pb.fm_torus(32, 32, 16), precision=2)
    o = oracle.Oracle(pr)
    o.set_prims(pr.P)
    s = grmhd.Sim(pr)
    s.set_prims(pr.P)
    o.step(1)
    s.step(1)
    compare(s.get_prims(), o.get_prims(), tol=TOL_FF, what="drift ff", rule="group")
    assert np.array_equal(s.flags()[0], o.flags()[0])


def test_drift_only_changes_bounded_zones(grmhd):
    """The predictor's update is zone-local: the frames differ only where a
    bound added mass or energy."""
    base = pb.fm_torus(24, 24, 8)
    out = {}
    for frame in (0, 1):
        s = grmhd.Sim(dataclasses.replace(base, floor_frame=frame))
        s.set_prims(base.P)
        s.predictor()
        out[frame] = (s.get_prims(),) + s.flags()
        s.close()
    (Pf, pf_f, ff_f), (Pd, pf_d, ff_d) = out[0], out[1]
    assert np.array_equal(pf_f, pf_d)
    ok = pf_f == 0  # fixed-up zones average neighbours that may differ
    untouched = ok & (ff_f == 0) & (ff_d == 0)
    assert untouched.sum() > 0
    assert np.array_equal(Pf[:, untouched], Pd[:, untouched])
    # the frames agree on which zones need mass or energy
    need_f = (ff_f & ~1) != 0
    need_d = (ff_d & ~(1 | FF_DRIFT | FF_DRIFT_FAIL)) != 0
    assert np.array_equal(need_f[ok], need_d[ok])
    parcel = ok & ((ff_d & FF_DRIFT) != 0)
    assert parcel.sum() > 100
    # the velocity changes only in zones that took a parcel, and does there
    dv = np.abs(Pd[2:5] - Pf[2:5]).max(axis=0)
    assert not (dv[ok & ~parcel] > 0).any()
    assert (dv[parcel] > 0).any()


def test_drift_batch_and_decomp_bitwise(grmhd):
    pr = _drift(pb.fm_torus(24, 20, 8))
    other = pb.fm_torus(20, 16, 4, recon=pb.RECON_MC)
    s = grmhd.Sim(pr)
    s.set_prims(pr.P)
    s.step(3)
    ref = s.get_prims(with_ghosts=True)
    s.close()
    sims = []
    for p in (other, pr):
        q = grmhd.Sim(p)
        q.set_prims(p.P)
        sims.append(q)
    b = grmhd.Batch(sims)
    b.step(3, sync=True)
    assert np.array_equal(sims[1].get_prims(with_ghosts=True), ref)
    b.close()
    for q in sims:
        q.close()
    d = grmhd.Decomp(pr, (2, 2, 2))
    d.set_prims(pr.P)
    d.step(3)
    assert np.array_equal(d.get_prims(with_ghosts=True), ref)
    d.close()


def test_drift_frame_validated(grmhd):
    with pytest.raises(Exception):
        grmhd.Sim(dataclasses.replace(pb.fm_torus(8, 8, 4), floor_frame=2))


def test_drift_full_size_torus_one_step(grmhd):
    """The bench's drift-frame workload, the 128^3 WENO5 torus: one step,
    every zone against the oracle at the FP64 bar."""
    pr = _drift(pb.fm_torus(128, 128, 128))
    o, s = _pair(pr, grmhd)
    o.step(1)
    s.step(1)
    compare(s.get_prims(), o.get_prims(), what="128^3 drift", ref=o)
    assert np.array_equal(s.flags()[0], o.flags()[0])
