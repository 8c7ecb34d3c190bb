"""Failure paths driven from the host with deliberately unphysical input
(negative internal energy in a few zones of the Orszag-Tang vortex, which
keeps every signal speed finite because the field dominates): the 1D_W
inversion fails there (u < 0), the fixup replaces the failed zones by their
neighbours' mean, and a failed zone whose every neighbour failed is reported
(GRMHD_ERR_INVERSION) while the step still completes -- all as the oracle
does.  Nothing here can fault the device: the state only changes values."""
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


def _planted(block):
    pr = pb.orszag_tang(32, recon=pb.RECON_WENO5)
    P = pr.P.copy()
    u0 = np.abs(P[1]).mean()
    if block:
        P[1, 0, 10:13, 10:13] = -u0  # the centre has no valid neighbour
    else:
        for (j, i) in ((5, 7), (20, 11), (13, 27)):
            P[1, 0, j, i] = -u0
    return pr, P


def _pair(grmhd, pr, P):
    o = oracle.Oracle(pr)
    o.set_prims(P)
    s = grmhd.Sim(pr)
    for loc in range(4):
        s.set_geom(loc, o.geom(loc))
    s.set_prims(P)
    return o, s


def test_planted_failures_are_fixed_up_as_the_oracle_does(grmhd):
    pr, P = _planted(block=False)
    o, s = _pair(grmhd, pr, P)
    o.predictor()
    s.predictor()
    pfo, _ = o.flags()
    pfg, _ = s.flags()
    assert (pfo == 5).sum() == 3  # u < 0 after the inversion
    assert np.array_equal(pfg, pfo)
    compare(s.get_prims(), o.get_prims(), what="fixup", ref=o)
    assert s.stats()["inv_failures"] == o.counters()["inv_failures"]


def test_unrecoverable_zone_is_reported_and_the_step_completes(grmhd):
    pr, P = _planted(block=True)
    o, s = _pair(grmhd, pr, P)
    assert o.step(1) == -4
    with pytest.raises(grmhd.GrmhdError) as e:
        s.step(1)
    assert e.value.code == -4  # GRMHD_ERR_INVERSION
    st, co = s.stats(), o.counters()
    assert st["unrecoverable"] == co["unrecoverable"] >= 1
    assert st["inv_failures"] == co["inv_failures"]
    assert st["steps"] == 1 and st["t"] == pytest.approx(o.time()[0], rel=1e-14)
    compare(s.get_prims(), o.get_prims(), what="unrecoverable", ref=o)
    # the error is reported once: the next clean step succeeds
    st2 = s.step(1)
    assert st2["steps"] == 2
