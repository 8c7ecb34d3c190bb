"""Domain decomposition (grmhd_decomp_*): the evolution of a grid split into
blocks is bitwise that of the undecomposed grid -- the paper's
decomposition tests -- for every boundary kind (periodic seams, X1
outflow, polar axis, fixed Bondi ghosts), both reconstructions, the flat
2D path, all four precision modes, and failed zones fixed up across block
edges."""
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


def _input(pr):
    Pg = pr.info.get("P_ghost") if pr.info else None
    return Pg if Pg is not None else pr.P


def _whole(grmhd, pr, n):
    s = grmhd.Sim(pr)
    s.set_prims(_input(pr))
    s.step(n, sync=False)
    st = s.stats()
    out = s.get_prims(with_ghosts=True)
    s.close()
    return out, st


def _split(grmhd, pr, nb, n):
    d = grmhd.Decomp(pr, nb)
    d.set_prims(_input(pr))
    st = d.step(n)
    out = d.get_prims(with_ghosts=True)
    d.close()
    return out, st


def _case(name):
    if name == "torus222":
        return pb.fm_torus(24, 20, 8), (2, 2, 2), 3
    if name == "torus_mc_x1":
        return pb.fm_torus(24, 20, 8, recon=pb.RECON_MC), (3, 1, 1), 3
    if name == "torus_x2x3":
        return pb.fm_torus(24, 20, 8), (1, 3, 2), 2
    if name == "mode2d":
        return pb.linear_mode(32, kind="alfven", amp=1e-3), (2, 2, 1), 4
    if name == "ot":
        return pb.orszag_tang(24, recon=pb.RECON_WENO5), (2, 3, 1), 3
    if name == "bondi":
        return pb.bondi(32, 24), (2, 2, 1), 3
    if name == "torus_mixed":
        pr = pb.fm_torus(24, 20, 8)
        pr.precision = 1
        return pr, (2, 2, 1), 2
    if name == "torus_ff":
        pr = pb.fm_torus(24, 20, 8)
        pr.precision = 2
        return pr, (1, 2, 2), 2
    if name == "torus_mixed_ff":
        pr = pb.fm_torus(24, 20, 8)
        pr.precision = 3
        return pr, (2, 1, 2), 2
    raise KeyError(name)


@pytest.mark.parametrize("name", ["torus222", "torus_mc_x1", "torus_x2x3", "mode2d", "ot", "bondi",
                                  "torus_mixed", "torus_ff", "torus_mixed_ff"])
def test_decomposition_bitwise(grmhd, name):
    pr, nb, n = _case(name)
    a, sa = _whole(grmhd, pr, n)
    b, sb = _split(grmhd, pr, nb, n)
    assert np.array_equal(a, b), (name, np.argwhere(a != b)[:5])
    for key in ("t", "dt", "steps", "inv_failures", "floor_hits", "unrecoverable"):
        assert sa[key] == sb[key], (name, key, sa[key], sb[key])


def test_decomposition_fixes_up_across_edges(grmhd):
    """The torus steps above do fix up failed zones; at least one of them
    sits next to a block edge, so the one-layer exchange before the fixup
    is exercised."""
    pr, nb, n = _case("torus222")
    s = grmhd.Sim(pr)
    s.set_prims(pr.P)
    s.step(1, sync=False)
    pf, _ = s.flags()
    s.close()
    assert pf.any()
    n3, n2, n1 = pf.shape
    edges = np.zeros_like(pf, dtype=bool)
    edges[:, :, n1 // 2 - 1:n1 // 2 + 1] = True
    edges[:, n2 // 2 - 1:n2 // 2 + 1, :] = True
    edges[n3 // 2 - 1:n3 // 2 + 1, :, :] = True
    assert (pf.astype(bool) & edges).any()


def test_decomposition_rejects_thin_blocks(grmhd):
    pr = pb.fm_torus(24, 20, 8)
    with pytest.raises(grmhd.GrmhdError):
        grmhd.Decomp(pr, (1, 1, 3))   # 8 / 3 < 3 zones per block
    with pytest.raises(grmhd.GrmhdError):
        grmhd.Decomp(pr, (0, 1, 1))
