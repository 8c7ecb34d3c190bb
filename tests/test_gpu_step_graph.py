"""grmhd_step replays a CUDA graph of one cycle when asked for several
cycles with profiling off: bitwise the cycles launched one by one (profiling
on takes the direct path), with the same launch counts, ordered with the
simulation's stream, and rebuilt after the autotuner changes the launch
shapes."""
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


@pytest.mark.parametrize("make", [lambda: pb.fm_torus(24, 20, 8), lambda: pb.linear_mode(32),
                                  lambda: pb.with_electrons(pb.fm_torus(20, 16, 8),
                                                            model=pb.ELEC_KAWAZURA)])
def test_graph_steps_bitwise_direct(grmhd, make):
    pr = make()
    out = []
    for graph in (True, False):
        s = grmhd.Sim(pr)
        s.set_prims(pr.P)
        if pr.electrons:
            s.set_electrons(pr.K)
        if graph:
            st = s.step(5)  # one call of several cycles: the graph
        else:
            s.profile(True)  # profiling forces direct launches
            for _ in range(5):
                st = s.step(1)
        prof = s.get_profile(reset=True)
        out.append((s.get_prims(with_ghosts=True), st, {k: v[1] for k, v in prof.items()},
                    s.get_electrons(with_ghosts=True) if pr.electrons else None))
        s.close()
    (Pg, sg, lg, Kg), (Pd, sd, ld, Kd) = out
    assert np.array_equal(Pg, Pd)
    if Kg is not None:
        assert np.array_equal(Kg, Kd)
    for key in ("t", "dt", "steps", "inv_failures", "floor_hits"):
        assert sg[key] == sd[key], key
    assert lg == ld  # the same kernels, counted per class


def test_graph_after_autotune_and_mixed_calls(grmhd):
    pr = pb.fm_torus(24, 20, 8)
    a = grmhd.Sim(pr)
    a.set_prims(pr.P)
    a.step(2)  # graph captured
    a.autotune(trials=1)  # new launch shapes: the graph is rebuilt
    a.step(1)
    a.step(3)
    b = grmhd.Sim(pr)
    b.set_prims(pr.P)
    for _ in range(6):
        b.step(1)
    assert np.array_equal(a.get_prims(with_ghosts=True), b.get_prims(with_ghosts=True))
    a.close()
    b.close()
