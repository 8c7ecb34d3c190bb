"""The FP64 reconstruction's walk length changes only the launch shape. One
thread walks 2, 4, 8 or 16 zones of a column and shares each zone's stencil
differences with the next. The X1 walk stages each warp's rows in shared
memory. Either way the face values, and so every cycle, are bitwise those
of one thread per zone (WENO5 pair of the "Implementation Notes"; MC too).

The grids here are small, so the automatic choice is one thread per zone;
each length is forced with grmhd_set_recon_walk. The 128^3 workload runs
the 16-zone walk by default; tests/test_gpu_parity.py::
test_full_size_torus_one_step checks it against the oracle zone by zone."""
import numpy as np
import pytest

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


def _run(grmhd, pr, rw, cycles):
    s = grmhd.Sim(pr)
    assert s.set_recon_walk(rw) == rw
    s.set_prims(pr.P)
    if pr.electrons:
        s.set_electrons(pr.K)
    s.step(cycles)
    out = (s.get_prims(with_ghosts=True), s.stats(), s.fluxes()[0])
    s.close()
    return out


@pytest.mark.parametrize("make", [
    lambda: pb.fm_torus(13, 11, 7),  # ragged: segments of every length, warps across rows
    lambda: pb.fm_torus(37, 21, 9),  # X1 longer than 32: two full 16-zone segments and a tail
    lambda: pb.fm_torus(24, 20, 8, recon=pb.RECON_MC),
    lambda: pb.orszag_tang(48, recon=pb.RECON_WENO5),  # flat X3
    lambda: pb.with_electrons(pb.fm_torus(20, 16, 8), model=pb.ELEC_KAWAZURA),
])
def test_walk_lengths_bitwise(grmhd, make):
    pr = make()
    P1, st1, F1 = _run(grmhd, pr, 1, 3)
    for rw in (2, 4, 8, 16):
        P, st, F = _run(grmhd, pr, rw, 3)
        assert np.array_equal(P, P1), rw
        assert np.array_equal(F, F1), rw
        for key in ("t", "dt", "steps", "inv_failures", "floor_hits"):
            assert st[key] == st1[key], (rw, key)


def test_walk_length_choice_and_errors(grmhd):
    pr = pb.fm_torus(24, 20, 8)
    s = grmhd.Sim(pr)
    # 26 x 22 x 10 zones cannot give a walk launch 152 x 640 threads
    assert s.set_recon_walk(0) == 1
    for bad in (3, 5, 17, 32, -1):
        with pytest.raises(RuntimeError):
            s.set_recon_walk(bad)
    assert s.set_recon_walk(8) == 8
    s.set_prims(pr.P)
    s.step(2)  # after a refused setting the plan still runs
    assert np.isfinite(s.get_prims()).all()
    s.close()


def test_walk_then_autotune_and_graph(grmhd):
    """The walk length and the tuner's block sizes compose; the replayed
    graph is rebuilt after either changes the launch shape."""
    pr = pb.fm_torus(37, 21, 9)
    ref, _, _ = _run(grmhd, pr, 1, 4)
    s = grmhd.Sim(pr)
    s.set_prims(pr.P)
    s.step(2)  # graph captured with the automatic choice
    s.set_recon_walk(16)
    s.autotune(trials=1)
    s.step(2)
    assert np.array_equal(s.get_prims(with_ghosts=True), ref)
    s.close()
