"""Pins of the oracle's fixup of failed zones and of the time step's growth
limit, each against values worked out here from the reading's own
definition (neither is printed in the paper; both come from the HARM
method the paper builds on).

Fixup reading: a zone whose 1D_W inversion failed takes, for rho, u and
utilde^1..3, the mean over the non-failed interior zones of its 3x3x3
neighbourhood (26 zones, itself excluded); B is kept; a zone with no valid
neighbour is reported as an error.  The cases plant zones with u < 0 in a
flat periodic box whose every other variable is a quadratic polynomial of
the coordinates, and run one step so short (t_final = 1e-30) that the
update leaves every zone where it was: the expected mean is then the mean
of the polynomial over the neighbour offsets, written out below
(26 neighbours: the quadratic term in direction d gains h^2 * 18/26).

Time-step reading: dt = min(CFL step, 1.3 dt_previous), the last step
landing on t_final.  With a tiny previous step the limit binds and the next
step is exactly 1.3 times it; with a large one the CFL step of the uniform
state (closed form) is taken.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2110_10191_gb300 import problems as pb

N = 9  # zones per side; the planted zones sit in the middle
H = 1.0 / N
GAM = 5.0 / 3.0
# coefficients (a, cx, cy, cz) of the quadratic fields of rho, u, utilde^1..3
COEF = {0: (1.0, 1.0, 2.0, 3.0), 1: (0.8, 0.5, 0.25, 0.75), 2: (0.0, 0.01, -0.01, 0.0),
        3: (0.0, 0.0, 0.02, 0.02), 4: (0.0, 0.01, 0.0, 0.02)}
B0 = (0.5, 0.3, 0.2)
U_FAIL = -0.05  # internal energy of a planted zone: the inversion recovers u < 0


def field(v, i, j, k):
    """The quadratic field of variable v (0..4) at zone (i, j, k)."""
    a, cx, cy, cz = COEF[v]
    x, y, z = (i + 0.5) * H, (j + 0.5) * H, (k + 0.5) * H
    return a + cx * x * x + cy * y * y + cz * z * z


def box(failed):
    """Flat periodic N^3 box with the quadratic fields, uniform B, and u < 0
    in the zones listed in `failed` ((i, j, k) tuples)."""
    P = np.zeros((8, N, N, N))
    k, j, i = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    for v in range(5):
        P[v] = field(v, i, j, k)
    for q in range(3):
        P[5 + q] = B0[q]
    for (fi, fj, fk) in failed:
        P[1, fk, fj, fi] = U_FAIL
    return pb.Problem(name="fixup box", n=(N, N, N), xmin=(0, 0, 0), xmax=(1, 1, 1), metric=0,
                      a=0.0, hslope=1.0, gamma=GAM, cfl=0.5, t_final=1e-30,
                      recon=pb.RECON_MC, floors=0, bc=((0, 0),) * 3, P=P)


def neighbour_mean(v, c, exclude=()):
    """Mean of field v over the 26 neighbours of zone c, without the zones
    in `exclude`, from the polynomial itself."""
    vals = []
    for dk in (-1, 0, 1):
        for dj in (-1, 0, 1):
            for di in (-1, 0, 1):
                z = (c[0] + di, c[1] + dj, c[2] + dk)
                if (di, dj, dk) == (0, 0, 0) or z in exclude:
                    continue
                vals.append(field(v, *z))
    return sum(vals) / len(vals), len(vals)


def run(failed):
    pr = box(failed)
    o = oracle.Oracle(pr)
    o.set_prims(pr.P)
    rc = o.step(1)
    return o, pr, rc


def test_fixup_is_the_mean_of_the_26_neighbours():
    c = (4, 4, 4)
    o, pr, rc = run([c])
    assert rc == 0
    assert o.time()[0] == 1e-30
    P = o.get_prims()
    pf, _ = o.flags()
    assert pf[c[2], c[1], c[0]] != 0 and int((pf != 0).sum()) == 1
    for v in range(5):
        exp, cnt = neighbour_mean(v, c)
        assert cnt == 26
        # closed form of the same mean: each quadratic term gains h^2 * 18/26
        a, cx, cy, cz = COEF[v]
        closed = field(v, *c) + (cx + cy + cz) * H * H * 18.0 / 26.0
        assert exp == pytest.approx(closed, rel=1e-14, abs=1e-16)
        assert P[v, c[2], c[1], c[0]] == pytest.approx(exp, rel=1e-12, abs=1e-15), v
    # B is kept, and every other zone is where it was
    for q in range(3):
        assert P[5 + q, c[2], c[1], c[0]] == pytest.approx(B0[q], rel=1e-14)
    mask = np.ones((N, N, N), bool)
    mask[c[2], c[1], c[0]] = False
    assert np.allclose(P[:, mask], pr.P[:, mask], rtol=1e-13, atol=1e-16)


def test_fixup_leaves_a_failed_neighbour_out():
    a, b = (4, 4, 4), (5, 4, 4)
    o, pr, rc = run([a, b])
    assert rc == 0
    P = o.get_prims()
    for c, other in ((a, b), (b, a)):
        for v in range(5):
            exp, cnt = neighbour_mean(v, c, exclude=(other,))
            assert cnt == 25
            assert P[v, c[2], c[1], c[0]] == pytest.approx(exp, rel=1e-12, abs=1e-15), (c, v)


def test_fixup_without_a_valid_neighbour_is_an_error():
    block = [(i, j, k) for k in (3, 4, 5) for j in (3, 4, 5) for i in (3, 4, 5)]
    o, pr, rc = run(block)
    assert rc == -4
    assert o.counters()["unrecoverable"] >= 1
    P = o.get_prims()
    # the centre keeps its own (failed) values; the block's other zones each
    # have valid neighbours outside the block and take their mean
    assert P[1, 4, 4, 4] == U_FAIL
    c = (3, 4, 4)
    exp, cnt = neighbour_mean(1, c, exclude=tuple(block))
    assert cnt == 9
    assert P[1, c[2], c[1], c[0]] == pytest.approx(exp, rel=1e-12)


def _uniform(cfl=0.9):
    P = np.empty((8, 4, 8, 16))
    for v, x in enumerate([1.0, 2.0, 0, 0, 0, 0.5, 0.3, -0.2]):
        P[v] = x
    return pb.Problem(name="uniform", n=(16, 8, 4), xmin=(0, 0, 0), xmax=(1, 1, 1), metric=0,
                      a=0.0, hslope=1.0, gamma=GAM, cfl=cfl, t_final=0.0,
                      recon=pb.RECON_WENO5, floors=0, bc=((0, 0),) * 3, P=P)


def _cfl_dt(cfl=0.9):
    """CFL step of the uniform state: c_ms of rho = 1, u = 2, B = (0.5, 0.3,
    -0.2) at rest, dt = 1 / sum_d(c_ms / (cfl dx_d))."""
    ef = 1 + GAM * 2.0
    bsq = 0.25 + 0.09 + 0.04
    cs2 = GAM * (GAM - 1) * 2.0 / ef
    va2 = bsq / (bsq + ef)
    c = math.sqrt(cs2 + va2 - cs2 * va2)
    return 1.0 / sum(c / (cfl * d) for d in (1 / 16, 1 / 8, 1 / 4))


def test_dt_growth_is_limited_to_1_3_of_the_previous_step():
    pr = _uniform()
    o = oracle.Oracle(pr)
    o.set_prims(pr.P)
    cfl_dt = _cfl_dt()
    for prev in (1e-6, 0.25 * cfl_dt, cfl_dt / 1.3 * 0.999):
        o.set_time(0.0, prev, 1)
        assert o.next_dt() == 1.3 * prev, prev
    # the limit does not bind: the CFL step
    for prev in (cfl_dt / 1.3 * 1.001, cfl_dt, 10.0):
        o.set_time(0.0, prev, 1)
        assert o.next_dt() == pytest.approx(cfl_dt, rel=1e-14), prev
    # no previous step (the first one): no limit
    o.set_time(0.0, 0.0, 0)
    assert o.next_dt() == pytest.approx(cfl_dt, rel=1e-14)


def test_dt_growth_limit_carries_through_steps():
    """Stepping from a tiny previous step: each step is 1.3 times the last
    until the CFL step binds."""
    pr = _uniform()
    o = oracle.Oracle(pr)
    o.set_prims(pr.P)
    cfl_dt = _cfl_dt()
    prev = 1e-3 * cfl_dt
    o.set_time(0.0, prev, 1)
    t = 0.0
    for _ in range(40):
        o.step(1)
        t_new, dt, _ = o.time()
        want = min(1.3 * prev, cfl_dt)
        assert dt == pytest.approx(want, rel=1e-14)
        assert t_new == pytest.approx(t + want, rel=1e-14)
        t, prev = t_new, dt
    assert dt == pytest.approx(cfl_dt, rel=1e-14)
