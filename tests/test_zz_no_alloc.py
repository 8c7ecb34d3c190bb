"""grmhd_fluxes_noalloc: the flux stage for callers that cannot allocate
device memory (it keeps its intermediates in a fixed file-scope device
array).  Its output must equal the regular path's (grmhd_get_fluxes on a
simulation holding the same state) within the flux tolerance of the parity
tests, on two calls in a row that share the array.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

from paper_2110_10191_gb300 import problems as pb

pytestmark = pytest.mark.gpu


def _check_close(Fn, Fr, tol=1e-12):
    for d in range(3):
        for grp in ((0, 1, 2, 3, 4), (5, 6, 7)):
            sc = max(np.abs(Fr[d, v]).max() for v in grp)
            for v in grp:
                assert np.abs(Fn[d, v] - Fr[d, v]).max() <= tol * max(sc, 1e-300), (d, v)


def test_fluxes_noalloc_matches_regular_path_twice():
    import torch
    from paper_2110_10191_gb300 import grmhd
    assert torch.cuda.is_available()
    cases = [pb.fm_torus(24, 20, 6, recon=pb.RECON_WENO5),
             pb.orszag_tang(40, recon=pb.RECON_MC)]
    for pr in cases:  # two calls in a row, different grids, same scratch
        sim = grmhd.Sim(pr)
        sim.set_prims(pr.P)
        Pg = torch.from_numpy(sim.get_prims(with_ghosts=True)).cuda()
        F_ref, ct_ref = sim.fluxes()
        F = torch.full((3, 8) + tuple(Pg.shape[1:]), 7.0, dtype=torch.float64, device="cuda")
        ct = grmhd.fluxes_noalloc(pr, Pg, F)
        torch.cuda.synchronize()
        _check_close(F.cpu().numpy(), F_ref)
        assert np.allclose(ct, ct_ref, rtol=1e-13, atol=0)
        sim.close()


def test_fluxes_noalloc_scratch_limit():
    """The largest cube the fixed scratch holds (123^3: 24 N + 936 A bytes
    plus alignment within 64 MiB) runs and matches the regular path; the
    next one (124^3) and far larger grids are refused."""
    import torch
    from paper_2110_10191_gb300 import grmhd
    pr = pb.fm_torus(123, 123, 123, recon=pb.RECON_WENO5)
    sim = grmhd.Sim(pr)
    sim.set_prims(pr.P)
    Pg = torch.from_numpy(sim.get_prims(with_ghosts=True)).cuda()
    F_ref, ct_ref = sim.fluxes()
    sim.close()
    F = torch.empty((3, 8) + tuple(Pg.shape[1:]), dtype=torch.float64, device="cuda")
    ct = grmhd.fluxes_noalloc(pr, Pg, F)
    torch.cuda.synchronize()
    _check_close(F.cpu().numpy(), F_ref)
    assert np.allclose(ct, ct_ref, rtol=1e-13, atol=0)
    del F, Pg
    P = torch.zeros(1, dtype=torch.float64, device="cuda")
    for n in ((124, 124, 124), (400, 400, 400)):
        big = pb.linear_mode(8)
        big.n = n
        with pytest.raises(grmhd.GrmhdError) as e:
            grmhd.fluxes_noalloc(big, P, P)
        assert e.value.code == -1, n
