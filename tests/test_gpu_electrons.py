"""Electron entropies on the GPU (grmhd_params.electrons) against the
oracle's electron thermodynamics.

* One step of the Kerr torus with each heating model (and the constant
  share): primitives within the FP64 one-step bar (1e-12 of each group's
  scale, 1e-9 per zone), the two entropies within the same bar of their own
  scales, failure codes exactly, bound flags but for knife edges.
* MC and WENO5, drift-frame bounds, the predictor alone, and the Bondi
  problem whose FIXED ghosts carry set entropies.
* With no electron heating the electron entropy is conserved on a periodic
  grid; batched grids with electrons are bitwise the grids alone.
* Every precision mode evolves them: float-float grids within that mode's
  bar (3e-11) of the oracle, the FP32-flux modes within the mixed mode's
  (1e-5); batches mixing the modes stay bitwise.
* Decomposed grids exchange the entropies: bitwise the whole grid's.
* Served requests carry them (grmhd_server_submit_electrons): bitwise the
  simulation alone.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_2110_10191_gb300 import problems as pb

from test_gpu_parity import compare

pytestmark = pytest.mark.gpu

MODELS = [pb.ELEC_CONSTANT, pb.ELEC_KAWAZURA, pb.ELEC_WERNER, pb.ELEC_ROWAN, pb.ELEC_SHARMA,
          pb.ELEC_HOWES]


@pytest.fixture(scope="module")
def grmhd():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2110_10191_gb300 import grmhd as g
    g.load()
    return g


def _pair(pr, grmhd, shared_geometry=True):
    o = oracle.Oracle(pr)
    Pg = pr.info.get("P_ghost") if pr.info else None
    Kg = pr.info.get("K_ghost") if pr.info else None
    o.set_prims(Pg if Pg is not None else pr.P)
    o.set_K(Kg if Kg is not None else pr.K)
    s = grmhd.Sim(pr)
    if shared_geometry:
        for loc in range(4):
            s.set_geom(loc, o.geom(loc))
    s.set_prims(Pg if Pg is not None else pr.P)
    s.set_electrons(Kg if Kg is not None else pr.K)
    return o, s


def compare_K(a, b, tol=1e-12, tol_zone=1e-9, what=""):
    for q in range(2):
        sc = np.abs(b[q]).max()
        d = np.abs(a[q] - b[q])
        assert d.max() <= tol * sc, (what, q, d.max() / sc)
        assert not (d > tol_zone * np.abs(b[q]) + tol * sc).any(), (what, q)


def _check_step(o, s, what, ff_slack=True):
    compare(s.get_prims(), o.get_prims(), what=what, ref=o)
    compare_K(s.get_electrons(), o.get_K(), what=what)
    pfo, ffo = o.flags()
    pfg, ffg = s.flags()
    assert np.array_equal(pfg, pfo), what
    mism = ffg != ffo
    assert mism.sum() <= max(2, ffo.size // 10000), (what, int(mism.sum()))


@pytest.mark.parametrize("model", MODELS)
def test_electron_step_parity_models(grmhd, model):
    pr = pb.with_electrons(pb.fm_torus(24, 20, 8), model=model)
    o, s = _pair(pr, grmhd)
    o.step(1)
    st = s.step(1)
    _check_step(o, s, "model %d" % model)
    co = o.counters()
    assert st["inv_failures"] == co["inv_failures"]
    assert abs(st["floor_hits"] - co["floor_hits"]) <= 2


@pytest.mark.parametrize("shape,recon,frame", [((32, 32, 16), pb.RECON_WENO5, 0),
                                               ((24, 20, 8), pb.RECON_MC, 0),
                                               ((24, 20, 8), pb.RECON_WENO5, 1),
                                               ((32, 32, 1), pb.RECON_WENO5, 0)])
def test_electron_step_parity_torus(grmhd, shape, recon, frame):
    pr = pb.with_electrons(dataclasses.replace(pb.fm_torus(*shape, recon=recon), floor_frame=frame),
                           model=pb.ELEC_KAWAZURA)
    o, s = _pair(pr, grmhd)
    o.step(2)
    s.step(2)
    # two steps: the second starts from states that already differ by rounding
    compare(s.get_prims(), o.get_prims(), tol=1e-11, what=str(shape), ref=o)
    compare_K(s.get_electrons(), o.get_K(), tol=1e-11, what=str(shape))
    assert np.array_equal(s.flags()[0], o.flags()[0])


def test_electron_predictor_parity(grmhd):
    pr = pb.with_electrons(pb.fm_torus(24, 24, 8), model=pb.ELEC_HOWES)
    o, s = _pair(pr, grmhd)
    o.predictor()
    s.predictor()
    _check_step(o, s, "predictor")


def test_electron_bondi_fixed_ghosts(grmhd):
    pr = pb.with_electrons(pb.bondi(32, 24, n3=2, recon=pb.RECON_WENO5), model=pb.ELEC_WERNER)
    o, s = _pair(pr, grmhd)
    o.step(3)
    s.step(3)
    compare(s.get_prims(), o.get_prims(), tol=1e-11, what="bondi", ref=o)
    compare_K(s.get_electrons(), o.get_K(), tol=1e-11, what="bondi")
    Kg = s.get_electrons(with_ghosts=True)
    assert np.array_equal(Kg[:, :, :, :3], pr.info["K_ghost"][:, :, :, :3])


def test_electron_entropy_conserved_without_heating(grmhd):
    pr = pb.with_electrons(pb.orszag_tang(48, recon=pb.RECON_WENO5), model=pb.ELEC_CONSTANT,
                           fel=0.0, tpte_min=0.0, tpte_max=math.inf)
    n = pr.n[0]
    x = (np.arange(n) + 0.5) / n
    K = pr.K.copy()
    K[1] *= 1 + 0.5 * np.sin(2 * np.pi * x)[None, None, :] * np.cos(2 * np.pi * x)[None, :, None]
    s = grmhd.Sim(pr)
    s.set_prims(pr.P)
    s.set_electrons(K)

    def total():
        P, Kn = s.get_prims(), s.get_electrons()
        gam = np.sqrt(1 + (P[2:5] ** 2).sum(axis=0))
        return float((P[0] * gam * Kn[1]).sum())

    k0 = total()
    s.step(10)
    assert total() == pytest.approx(k0, rel=1e-13)
    assert not np.allclose(s.get_electrons()[1], K[1], rtol=1e-6, atol=0)


def test_electron_batch_bitwise(grmhd):
    probs = [pb.with_electrons(pb.fm_torus(24, 20, 8), model=pb.ELEC_ROWAN),
             pb.fm_torus(20, 16, 4, recon=pb.RECON_MC),
             pb.with_electrons(pb.orszag_tang(32, recon=pb.RECON_WENO5), model=pb.ELEC_SHARMA)]
    ref = []
    for pr in probs:
        s = grmhd.Sim(pr)
        s.set_prims(pr.P)
        if pr.electrons:
            s.set_electrons(pr.K)
        s.step(3)
        ref.append((s.get_prims(with_ghosts=True),
                    s.get_electrons(with_ghosts=True) if pr.electrons else None))
        s.close()
    sims = []
    for pr in probs:
        s = grmhd.Sim(pr)
        s.set_prims(pr.P)
        if pr.electrons:
            s.set_electrons(pr.K)
        sims.append(s)
    b = grmhd.Batch(sims)
    b.step(3, sync=True)
    for s, pr, (P, K) in zip(sims, probs, ref):
        assert np.array_equal(s.get_prims(with_ghosts=True), P), pr.name
        if K is not None:
            assert np.array_equal(s.get_electrons(with_ghosts=True), K), pr.name
    b.close()
    for s in sims:
        s.close()


@pytest.mark.parametrize("prec,tol", [(2, 3e-11), (1, 1e-5), (3, 1e-5)])
def test_electron_step_parity_precisions(grmhd, prec, tol):
    pr = dataclasses.replace(pb.with_electrons(pb.fm_torus(32, 32, 16), model=pb.ELEC_KAWAZURA),
                             precision=prec)
    o, s = _pair(pr, grmhd)
    o.step(1)
    s.step(1)
    compare(s.get_prims(), o.get_prims(), tol=tol, what="precision %d" % prec,
            rule="group")
    # kappa_tot = (gamma - 1) u / rho^gamma carries the relative errors of u
    # and gamma times those of rho, and peaks in hot, thin zones whose u is far
    # below the group scale the primitives' bar refers to: with FP32 fluxes
    # its bar is ten times the primitives' (measured 1.2e-5 of max kappa)
    ktol = tol if prec == 2 else 10 * tol
    compare_K(s.get_electrons(), o.get_K(), tol=ktol, tol_zone=max(1e-9, ktol),
              what="precision %d" % prec)
    if prec == 2:
        assert np.array_equal(s.flags()[0], o.flags()[0])


def test_electron_batch_of_all_precisions(grmhd):
    probs = [dataclasses.replace(pb.with_electrons(pb.fm_torus(20, 16, 8), model=m), precision=q)
             for q, m in enumerate((pb.ELEC_HOWES, pb.ELEC_WERNER, pb.ELEC_ROWAN, pb.ELEC_SHARMA))]
    ref = []
    for pr in probs:
        s = grmhd.Sim(pr)
        s.set_prims(pr.P)
        s.set_electrons(pr.K)
        s.step(2)
        ref.append((s.get_prims(with_ghosts=True), s.get_electrons(with_ghosts=True)))
        s.close()
    sims = []
    for pr in probs:
        s = grmhd.Sim(pr)
        s.set_prims(pr.P)
        s.set_electrons(pr.K)
        sims.append(s)
    b = grmhd.Batch(sims)
    b.step(2, sync=True)
    for s, pr, (P, K) in zip(sims, probs, ref):
        assert np.array_equal(s.get_prims(with_ghosts=True), P), pr.precision
        assert np.array_equal(s.get_electrons(with_ghosts=True), K), pr.precision
    b.close()
    for s in sims:
        s.close()


@pytest.mark.parametrize("nb,prec", [((2, 2, 2), 0), ((1, 3, 2), 3)])
def test_electron_decomposition_bitwise(grmhd, nb, prec):
    """Blocks exchange the entropies with the primitives: the decomposed
    evolution is bitwise the whole grid's, entropies included."""
    pr = dataclasses.replace(pb.with_electrons(pb.fm_torus(24, 20, 8), model=pb.ELEC_KAWAZURA),
                             precision=prec)
    s = grmhd.Sim(pr)
    s.set_prims(pr.P)
    s.set_electrons(pr.K)
    s.step(3)
    P, K = s.get_prims(with_ghosts=True), s.get_electrons(with_ghosts=True)
    st = s.stats()
    s.close()
    d = grmhd.Decomp(pr, nb)
    d.set_prims(pr.P)
    d.set_electrons(pr.K)
    sd = d.step(3)
    assert np.array_equal(d.get_prims(with_ghosts=True), P)
    assert np.array_equal(d.get_electrons(with_ghosts=True), K)
    assert sd["floor_hits"] == st["floor_hits"] and sd["inv_failures"] == st["inv_failures"]
    d.close()


def test_electron_refusals(grmhd):
    pr = pb.with_electrons(pb.fm_torus(12, 12, 4), model=pb.ELEC_KAWAZURA)
    bad = dict(pr.electrons, game=1.0)
    with pytest.raises(Exception):
        grmhd.Sim(dataclasses.replace(pr, electrons=bad))
    s = grmhd.Sim(pb.fm_torus(12, 12, 4))
    with pytest.raises(Exception):
        s.set_electrons(pr.K)
    s.close()
    # the plain submission refuses electron requests: the entropies must travel
    g, m, p = grmhd._structs(pr)
    with grmhd.Server() as srv:
        out = np.empty_like(pr.P)
        assert srv.L.grmhd_server_submit(srv.h, 1, grmhd.ctypes.byref(g), grmhd.ctypes.byref(m),
                                         grmhd.ctypes.byref(p), pr.P.ctypes.data, 0,
                                         out.ctypes.data, 0, 2, -1.0) == -1


def test_electron_requests_are_served_bitwise(grmhd):
    """Requests with electrons through the serving loop, batched with a
    request without them: each result (primitives and entropies) is bitwise
    the simulation's result alone."""
    probs = [pb.with_electrons(pb.fm_torus(20, 16, 8), model=pb.ELEC_HOWES),
             pb.fm_torus(16, 16, 4),
             pb.with_electrons(pb.orszag_tang(24, recon=pb.RECON_WENO5), model=pb.ELEC_WERNER)]
    steps = [3, 2, 4]
    ref = []
    for pr, n in zip(probs, steps):
        s = grmhd.Sim(pr)
        s.set_prims(pr.P)
        if pr.electrons:
            s.set_electrons(pr.K)
        s.step(n)
        ref.append((s.get_prims(), s.get_electrons() if pr.electrons else None))
        s.close()
    with grmhd.Server(quantum=2) as srv:
        for q, (pr, n) in enumerate(zip(probs, steps)):
            srv.submit(q, pr, n)
        srv.drain()
        res = {r["id"]: r for r in srv.poll(16)}
    for q, (P, K) in enumerate(ref):
        assert res[q]["status"] == 0
        assert np.array_equal(res[q]["P"], P)
        if K is not None:
            assert np.array_equal(res[q]["K"], K)
        else:
            assert res[q]["K"] is None


def test_electron_full_size_torus_one_step(grmhd):
    """The bench's electron workload, the 128^3 WENO5 torus with Kawazura
    heating: one step, every zone's primitives and entropies against the
    oracle at the FP64 bar."""
    pr = pb.with_electrons(pb.fm_torus(128, 128, 128), model=pb.ELEC_KAWAZURA)
    o, s = _pair(pr, grmhd)
    o.step(1)
    s.step(1)
    compare(s.get_prims(), o.get_prims(), what="128^3 electrons", ref=o)
    compare_K(s.get_electrons(), o.get_K(), what="128^3 electrons")
    assert np.array_equal(s.flags()[0], o.flags()[0])
