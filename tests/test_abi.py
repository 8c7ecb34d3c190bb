"""The C-ABI library builds, loads and exports every entry point that
include/grmhd.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(grmhd_[a-z0-9_]+)\s*\(", src))
    return names


def test_header_declares_entry_points():
    names = _declared()
    for must in ("grmhd_create", "grmhd_step", "grmhd_set_prims", "grmhd_get_prims",
                 "grmhd_destroy", "grmhd_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2110_10191_gb300 import build, grmhd
    build.build()
    L = ctypes.CDLL(build.LIB)
    missing = [n for n in sorted(_declared()) if not hasattr(L, n)]
    assert not missing, missing
    # the binding wraps exactly the declared set
    assert set(grmhd.EXPORTS) == _declared()


def test_strerror_without_gpu():
    from paper_2110_10191_gb300 import grmhd
    L = grmhd.load()
    assert L.grmhd_strerror(0) == b"ok"
    assert L.grmhd_strerror(-4) == b"failed zone with no valid neighbour"


def test_buffers_must_be_contiguous_float64():
    """The binding hands the library raw pointers to doubles: other dtypes
    and non-contiguous views are refused before any call."""
    import numpy as np
    from paper_2110_10191_gb300 import grmhd
    assert grmhd._ptr(np.zeros((2, 3)))[1] == 0
    with pytest.raises(ValueError):
        grmhd._ptr(np.zeros(3, dtype=np.float32))
    with pytest.raises(ValueError):
        grmhd._ptr(np.zeros((4, 4))[:, ::2])
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        grmhd._ptr(torch.zeros(3, dtype=torch.float32))
    assert grmhd._ptr(torch.zeros(3, dtype=torch.float64))[1] == 0


def test_fluxes_noalloc_checks_arguments_as_create_does():
    """The allocation-free flux stage refuses, before any CUDA call, what
    grmhd_create refuses: a Kerr spin |a| >= 1, an unpaired periodic side,
    outflow off X1 (the pointers are never read on these paths)."""
    import dataclasses
    from paper_2110_10191_gb300 import grmhd, problems as pb
    L = grmhd.load()
    dummy = ctypes.c_void_p(256)
    cases = [dataclasses.replace(pb.fm_torus(8, 8, 4), a=1.0),
             dataclasses.replace(pb.linear_mode(8), bc=((0, 1), (0, 0), (0, 0))),
             dataclasses.replace(pb.linear_mode(8), bc=((0, 0), (1, 1), (0, 0)))]
    for pr in cases:
        g, m, p = grmhd._structs(pr)
        rc = L.grmhd_fluxes_noalloc(ctypes.byref(g), ctypes.byref(m), ctypes.byref(p), dummy, dummy,
                                    None, None)
        assert rc == -1, pr.name
