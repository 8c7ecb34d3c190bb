"""Batched stepping of many independent grids (grmhd_batch_*) and the flat-X3
mode of 2D grids.

The bar is bitwise: a grid's state after n batched steps must equal its
state after n steps alone (same kernels' bodies, one grid per block, per-grid
clock), whatever else shares the batch and with or without the CUDA graph.
The flat-X3 mode (n3 = 1, periodic X3) must equal the full-extent step, which
a grid with two identical X3 layers still runs.  Parity with the oracle is
checked per grid after one batched step at the FP64 tolerance of the
single-grid parity tests."""
import numpy as np
import pytest

import oracle
from paper_2110_10191_gb300 import problems as pb
from test_gpu_parity import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def grmhd():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2110_10191_gb300 import grmhd as g
    g.load()
    return g


def _mixture():
    """Eight uneven 2D grids of every kind plus two small tori (3D, outflow
    and polar boundaries, bounds on, both reconstructions)."""
    probs = pb.batch_2d(ngrid=8, nmin=12, nmax=40, seed=5)
    probs.append(pb.fm_torus(24, 20, 8))
    tor = pb.fm_torus(20, 16, 4)
    tor.recon = pb.RECON_MC
    probs.append(tor)
    return probs


def _alone(grmhd, pr, nsteps):
    s = grmhd.Sim(pr)
    s.set_prims(pr.P)
    st = s.step(nsteps)
    out = s.get_prims(with_ghosts=True)
    s.close()
    return out, st


def test_batch_with_walks_bitwise_equals_alone(grmhd):
    """A batch large enough for the reconstruction's column walks (six tori
    of three sizes, different perturbations, fields and reconstructions, with
    a 2D and a mixed-precision grid beside them: 2-zone walks) while each
    grid alone is too small for them and takes one thread per zone: every
    grid bitwise its state alone, the X1 walk's shared-memory staging
    included."""
    probs = [pb.fm_torus(40, 32, 24, seed=s) for s in range(3)]
    probs += [pb.fm_torus(64, 32, 16, seed=s) for s in range(2)]
    probs.append(pb.fm_torus(40, 40, 20, recon=pb.RECON_MC, beta=30.0))
    probs.append(pb.orszag_tang(64, recon=pb.RECON_WENO5))
    mixed = pb.orszag_tang(64, recon=pb.RECON_WENO5)
    mixed.precision = 1
    probs.append(mixed)
    nsteps = 2
    ref = [_alone(grmhd, pr, nsteps) for pr in probs]
    one = grmhd.Sim(probs[0])
    assert one.set_recon_walk(0) == 1  # alone: one thread per zone
    one.close()
    sims = []
    for pr in probs:
        s = grmhd.Sim(pr)
        s.set_prims(pr.P)
        sims.append(s)
    b = grmhd.Batch(sims)
    assert b.info()["recon_walk"] >= 2
    b.step(nsteps, graph=True, sync=True)
    for s, (P, st), pr in zip(sims, ref, probs):
        assert np.array_equal(s.get_prims(with_ghosts=True), P), pr.name
        assert s.stats()["t"] == st["t"], pr.name
    b.close()


@pytest.mark.parametrize("graph", [True, False])
def test_batch_bitwise_equals_alone(grmhd, graph):
    probs = _mixture()
    nsteps = 3
    ref = [_alone(grmhd, pr, nsteps) for pr in probs]
    sims = []
    for pr in probs:
        s = grmhd.Sim(pr)
        s.set_prims(pr.P)
        sims.append(s)
    b = grmhd.Batch(sims)
    b.step(1, graph=graph)
    b.step(nsteps - 1, graph=graph, sync=True)
    info = b.info()
    assert info["ngrid"] == len(probs)
    assert info["zones"] == sum(pr.zones for pr in probs)
    assert info["launches"] == nsteps * info["launches_per_step"]
    assert info["graph"] == int(graph)
    dts = set()
    for s, (P, st), pr in zip(sims, ref, probs):
        got = s.get_prims(with_ghosts=True)
        assert np.array_equal(got, P), pr.name
        gs = s.stats()
        assert gs["t"] == st["t"] and gs["dt"] == st["dt"] and gs["steps"] == nsteps, pr.name
        assert gs["inv_failures"] == st["inv_failures"] and gs["floor_hits"] == st["floor_hits"]
        dts.add(gs["dt"])
    assert len(dts) > 1  # every grid took its own time step
    b.close()


def test_batch_independent_of_company(grmhd):
    """A grid gives the same bits in a batch of one, a batch of all, and a
    batch in another order."""
    probs = pb.batch_2d(ngrid=6, nmin=10, nmax=30, seed=11)

    def run(order):
        sims = [grmhd.Sim(probs[g]) for g in order]
        for s, g in zip(sims, order):
            s.set_prims(probs[g].P)
        b = grmhd.Batch(sims)
        b.step(2, sync=True)
        out = {g: s.get_prims() for s, g in zip(sims, order)}
        b.close()
        return out

    together = run(list(range(6)))
    reverse = run(list(range(5, -1, -1)))
    for g in range(6):
        single = run([g])
        assert np.array_equal(single[g], together[g])
        assert np.array_equal(reverse[g], together[g])


def test_batch_per_grid_t_final(grmhd):
    """A grid whose t_final is reached stops there; the others go on."""
    probs = pb.batch_2d(ngrid=3, nmin=16, nmax=24, seed=2)
    sims = [grmhd.Sim(pr) for pr in probs]
    for s, pr in zip(sims, probs):
        s.set_prims(pr.P)
    dt0 = sims[0].next_dt()
    sims[0].close()
    probs[0].t_final = 2.5 * dt0
    sims[0] = grmhd.Sim(probs[0])
    sims[0].set_prims(probs[0].P)
    b = grmhd.Batch(sims)
    b.step(6, sync=True)
    st = [s.stats() for s in sims]
    assert st[0]["t"] == pytest.approx(probs[0].t_final, rel=1e-14) and st[0]["steps"] < 6
    assert st[1]["steps"] == 6 and st[2]["steps"] == 6
    ref, rst = _alone(grmhd, probs[0], 6)
    assert np.array_equal(sims[0].get_prims(with_ghosts=True), ref)
    assert rst["t"] == st[0]["t"]
    b.close()


def test_batch_oracle_parity(grmhd):
    """One batched step of every grid against the oracle (same geometry)."""
    probs = _mixture()
    sims, oracles = [], []
    for pr in probs:
        o = oracle.Oracle(pr)
        o.set_prims(pr.P)
        s = grmhd.Sim(pr)
        for loc in range(4):
            s.set_geom(loc, o.geom(loc))
        s.set_prims(pr.P)
        sims.append(s)
        oracles.append(o)
    b = grmhd.Batch(sims)
    b.step(1, sync=True)
    for s, o, pr in zip(sims, oracles, probs):
        o.step(1)
        compare(s.get_prims(), o.get_prims(), what=pr.name, ref=o)
    b.close()


def test_batch_graph_replay_matches_direct(grmhd):
    probs = pb.batch_2d(ngrid=4, nmin=16, nmax=32, seed=9)
    outs = []
    for graph in (True, False):
        sims = [grmhd.Sim(pr) for pr in probs]
        for s, pr in zip(sims, probs):
            s.set_prims(pr.P)
        b = grmhd.Batch(sims)
        b.step(4, graph=graph, sync=True)
        outs.append([s.get_prims() for s in sims])
        b.close()
    for a, c in zip(*outs):
        assert np.array_equal(a, c)


def test_batch_then_single_steps_ordered(grmhd):
    """Single-grid calls after a batched step see its result (stream order),
    and stepping on alone continues bitwise."""
    pr = pb.orszag_tang(20)
    ref, _ = _alone(grmhd, pr, 3)
    s = grmhd.Sim(pr)
    s.set_prims(pr.P)
    b = grmhd.Batch([s])
    b.step(2)          # no host sync
    s.step(1)          # ordered after the batch on the simulation's stream
    assert np.array_equal(s.get_prims(with_ghosts=True), ref)
    b.close()


def test_batch_rejects_bad_members(grmhd):
    pr = pb.linear_mode(8)
    s = grmhd.Sim(pr)
    with pytest.raises(grmhd.GrmhdError):
        grmhd.Batch([s, s])
    with pytest.raises(grmhd.GrmhdError):
        grmhd.Batch([])


def test_batch_mixed_precision_members(grmhd):
    """Grids of all four precision modes in one batch: each bitwise its
    alone result (each flux and update kernel runs only on its own grids'
    blocks)."""
    probs = pb.batch_2d(ngrid=7, nmin=12, nmax=32, seed=4)
    tor = pb.fm_torus(24, 20, 8)
    probs.append(tor)
    for q, pr in enumerate(probs):
        pr.precision = q % 4
    ref = [_alone(grmhd, pr, 2)[0] for pr in probs]
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


@pytest.mark.parametrize("kind", ["orszag_tang", "alfven"])
def test_flat_x3_equals_full_extent(grmhd, kind):
    """n3 = 1 (flat mode: fluxes on one layer, copied) against the same
    problem on two identical X3 layers of a very long X3 period (full
    extent: every layer reconstructed; the X3 signal speed then changes the
    time step by less than its last bit)."""
    if kind == "orszag_tang":
        pr = pb.orszag_tang(24, recon=pb.RECON_WENO5)
    else:
        pr = pb.linear_mode(20, kind="alfven", amp=1e-3, recon=pb.RECON_MC)
    ext = pb.Problem(**{**pr.__dict__})
    ext.n = (pr.n[0], pr.n[1], 2)
    ext.xmax = (pr.xmax[0], pr.xmax[1], 1.0e300)
    ext.P = np.concatenate([pr.P, pr.P], axis=1)
    flat, _ = _alone(grmhd, pr, 3)
    full, _ = _alone(grmhd, ext, 3)
    ng = 3
    for k in range(2):
        assert np.array_equal(full[:, ng + k, ng:-ng, ng:-ng], flat[:, ng, ng:-ng, ng:-ng]), k


def test_flat_x3_mixed_precision_matches_full_extent(grmhd):
    pr = pb.orszag_tang(24, recon=pb.RECON_WENO5)
    pr.precision = 1
    ext = pb.Problem(**{**pr.__dict__})
    ext.n = (pr.n[0], pr.n[1], 2)
    ext.xmax = (pr.xmax[0], pr.xmax[1], 1.0e300)
    ext.P = np.concatenate([pr.P, pr.P], axis=1)
    flat, _ = _alone(grmhd, pr, 2)
    full, _ = _alone(grmhd, ext, 2)
    for k in range(2):
        assert np.array_equal(full[:, 3 + k, 3:-3, 3:-3], flat[:, 3, 3:-3, 3:-3]), k


def _fresh(grmhd, probs):
    sims = []
    for pr in probs:
        s = grmhd.Sim(pr)
        s.set_prims(pr.P)
        sims.append(s)
    return sims


def test_launch_settings_do_not_change_bits(grmhd):
    """Every block size and block order of the heavy kernels gives the same
    bits (each thread computes the same zone or face whatever the launch
    shape)."""
    probs = pb.batch_2d(ngrid=5, nmin=12, nmax=36, seed=8)
    probs.append(pb.fm_torus(20, 16, 4))
    probs[1].precision = 1
    ref = [_alone(grmhd, pr, 2)[0] for pr in probs]
    for threads, order in ((64, 2), (256, 1), (96, 0), (160, 2), (256, 2)):
        sims = _fresh(grmhd, probs)
        b = grmhd.Batch(sims)
        for kc in ("recon", "flux", "update"):
            b.set_launch(kc, threads, order)
        b.step(2, sync=True)
        for s, P, pr in zip(sims, ref, probs):
            assert np.array_equal(s.get_prims(with_ghosts=True), P), (threads, order, pr.name)
        b.close()


def test_set_launch_rejects_bad_values(grmhd):
    s = grmhd.Sim(pb.linear_mode(8))
    b = grmhd.Batch([s])
    for kc, th, od in (("recon", 32, 0), ("recon", 100, 0), ("flux", 512, 0), ("update", 128, 3),
                       ("bounds", 128, 0)):
        with pytest.raises(grmhd.GrmhdError):
            b.set_launch(kc, th, od)
    b.close()


def test_batch_autotune_keeps_state_and_bits(grmhd):
    probs = _mixture()
    ref = [_alone(grmhd, pr, 2) for pr in probs]
    sims = _fresh(grmhd, probs)
    b = grmhd.Batch(sims)
    b.step(1, sync=True)
    before = [(s.get_prims(with_ghosts=True), s.stats()) for s in sims]
    ms0, ms1 = b.autotune(trials=2)
    assert ms0 > 0 and 0 < ms1 <= ms0 * 1.05
    assert b.info()["tuned"] == 1 and b.info()["graph"] == 0
    for s, (P, st) in zip(sims, before):
        assert np.array_equal(s.get_prims(with_ghosts=True), P)
        assert s.stats() == st
    b.step(1, sync=True)
    for s, (P, st), pr in zip(sims, ref, probs):
        assert np.array_equal(s.get_prims(with_ghosts=True), P), pr.name
        assert s.stats()["t"] == st["t"]
    b.close()


def test_sim_autotune_keeps_bits(grmhd):
    pr = pb.fm_torus(24, 20, 8)
    ref, st = _alone(grmhd, pr, 2)
    s = grmhd.Sim(pr)
    s.set_prims(pr.P)
    ms0, ms1 = s.autotune(trials=2)
    assert ms0 > 0 and ms1 > 0
    got = s.step(2)
    assert np.array_equal(s.get_prims(with_ghosts=True), ref)
    assert got["t"] == st["t"] and got["floor_hits"] == st["floor_hits"]


def test_full_batch_oracle_parity(grmhd):
    """The batch the benchmark times -- 64 uneven 2D grids, 32^2 to 256^2
    (seed 0), autotuned and stepped through its CUDA graph -- one step,
    every grid against the oracle at the single-grid FP64 rule."""
    probs = pb.batch_2d(ngrid=64, nmin=32, nmax=256, seed=0)
    sims, oracles = [], []
    for pr in probs:
        o = oracle.Oracle(pr)
        o.set_prims(pr.P)
        s = grmhd.Sim(pr)
        for loc in range(4):
            s.set_geom(loc, o.geom(loc))
        s.set_prims(pr.P)
        sims.append(s)
        oracles.append(o)
    b = grmhd.Batch(sims)
    b.autotune(trials=1)
    b.step(1, graph=True, sync=True)
    assert b.info()["tuned"] == 1 and b.info()["graph"] == 1
    for s, o, pr in zip(sims, oracles, probs):
        o.step(1)
        compare(s.get_prims(), o.get_prims(), what=pr.name, ref=o)
        o.close()
    b.close()
    for s in sims:
        s.close()
