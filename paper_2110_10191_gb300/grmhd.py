"""ctypes binding of libgrmhd.so (include/grmhd.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Host arrays are numpy float64; device arrays may be torch CUDA
tensors (their data_ptr() is passed with on_device=1), and a torch CUDA
stream may be passed as the simulation's stream.  There is no CPU
fallback: if the library is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

NPRIM = 8
NG = 3
GRMHD_OK = 0
ERRORS = {-1: "invalid argument", -2: "device allocation failed", -3: "CUDA runtime error",
          -4: "failed zone with no valid neighbour", -5: "no finite time step"}

_lock = threading.Lock()
_lib = None


class GrmhdError(RuntimeError):
    def __init__(self, code, where):
        super().__init__("%s: %s (%d)" % (where, ERRORS.get(code, "unknown error"), code))
        self.code = code


class grmhd_grid(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_int), ("n2", ctypes.c_int), ("n3", ctypes.c_int),
                ("x1min", ctypes.c_double), ("x1max", ctypes.c_double),
                ("x2min", ctypes.c_double), ("x2max", ctypes.c_double),
                ("x3min", ctypes.c_double), ("x3max", ctypes.c_double)]


class grmhd_metric(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("a", ctypes.c_double), ("hslope", ctypes.c_double)]


PREC_FP64, PREC_MIXED, PREC_FF, PREC_MIXED_FF = 0, 1, 2, 3
FLOOR_FLUID, FLOOR_DRIFT = 0, 1


class grmhd_electrons(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("game", ctypes.c_double), ("gamp", ctypes.c_double),
                ("fel", ctypes.c_double), ("tpte_min", ctypes.c_double), ("tpte_max", ctypes.c_double)]


class grmhd_params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("cfl", ctypes.c_double), ("t_final", ctypes.c_double),
                ("recon", ctypes.c_int), ("floors_on", ctypes.c_int),
                ("bc", (ctypes.c_int * 2) * 3), ("precision", ctypes.c_int),
                ("floor_frame", ctypes.c_int), ("electrons", grmhd_electrons)]


KCLASSES = ["flux", "dt", "ct", "update", "fixup", "bounds", "other", "recon"]


class grmhd_profile_data(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 8), ("launches", ctypes.c_longlong * 8)]


class grmhd_stats(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("dt", ctypes.c_double), ("steps", ctypes.c_longlong),
                ("inv_failures", ctypes.c_longlong), ("floor_hits", ctypes.c_longlong),
                ("unrecoverable", ctypes.c_longlong)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class grmhd_batch_info(ctypes.Structure):
    _fields_ = [("ngrid", ctypes.c_int), ("zones", ctypes.c_longlong),
                ("launches_per_step", ctypes.c_int), ("launches", ctypes.c_longlong),
                ("graph", ctypes.c_int), ("tuned", ctypes.c_int), ("recon_walk", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class grmhd_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("max_active_zones", ctypes.c_longlong),
                ("quantum", ctypes.c_int), ("use_graph", ctypes.c_int), ("policy", ctypes.c_int)]


class grmhd_server_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("status", ctypes.c_int), ("zones", ctypes.c_longlong),
                ("steps", ctypes.c_longlong), ("t_arrival", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double), ("stats", grmhd_stats)]


class grmhd_server_stats(ctypes.Structure):
    _fields_ = [("now", ctypes.c_double), ("submitted", ctypes.c_longlong),
                ("completed", ctypes.c_longlong), ("failed", ctypes.c_longlong),
                ("rounds", ctypes.c_longlong), ("zone_cycles", ctypes.c_double),
                ("busy_seconds", ctypes.c_double), ("bytes_in_use", ctypes.c_size_t),
                ("peak_bytes", ctypes.c_size_t), ("budget", ctypes.c_size_t),
                ("active", ctypes.c_int), ("pending", ctypes.c_int), ("peak_active", ctypes.c_int),
                ("launches", ctypes.c_longlong)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


EXPORTS = ["grmhd_create", "grmhd_destroy", "grmhd_set_prims", "grmhd_set_prims_ghost",
           "grmhd_get_prims", "grmhd_step", "grmhd_get_stats", "grmhd_set_time",
           "grmhd_predictor", "grmhd_get_fluxes", "grmhd_next_dt", "grmhd_get_flags",
           "grmhd_get_geometry", "grmhd_set_geometry", "grmhd_divb", "grmhd_profile", "grmhd_get_profile",
           "grmhd_fp64_peak", "grmhd_fluxes_noalloc", "grmhd_batch_create", "grmhd_batch_destroy",
           "grmhd_batch_step", "grmhd_batch_get_info", "grmhd_batch_sync", "grmhd_autotune",
           "grmhd_set_recon_walk",
           "grmhd_batch_autotune", "grmhd_batch_set_launch", "grmhd_footprint", "grmhd_server_create",
           "grmhd_server_submit", "grmhd_server_poll", "grmhd_server_drain", "grmhd_server_get_stats",
           "grmhd_server_now", "grmhd_server_destroy", "grmhd_decomp_create", "grmhd_decomp_destroy",
           "grmhd_decomp_set_prims", "grmhd_decomp_get_prims", "grmhd_decomp_step",
           "grmhd_decomp_get_stats", "grmhd_set_electrons", "grmhd_get_electrons",
           "grmhd_decomp_set_electrons", "grmhd_decomp_get_electrons",
           "grmhd_server_submit_electrons", "grmhd_arith", "grmhd_fp64_probe",
           "grmhd_strerror"]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libgrmhd.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and not _build.up_to_date():
            _build.build()
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libgrmhd.so is not built (%s); run paper_2110_10191_gb300.build" % path)
        L = ctypes.CDLL(path)
        vp, i, d, P = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.POINTER
        L.grmhd_create.argtypes = [P(grmhd_grid), P(grmhd_metric), P(grmhd_params), vp, P(vp)]
        L.grmhd_destroy.argtypes = [vp]
        L.grmhd_set_prims.argtypes = [vp, vp, i]
        L.grmhd_set_prims_ghost.argtypes = [vp, vp, i]
        L.grmhd_get_prims.argtypes = [vp, vp, i, i]
        L.grmhd_set_electrons.argtypes = [vp, vp, i, i]
        L.grmhd_get_electrons.argtypes = [vp, vp, i, i]
        L.grmhd_step.argtypes = [vp, i, P(grmhd_stats)]
        L.grmhd_get_stats.argtypes = [vp, P(grmhd_stats)]
        L.grmhd_set_time.argtypes = [vp, d, d, ctypes.c_longlong]
        L.grmhd_predictor.argtypes = [vp]
        L.grmhd_get_fluxes.argtypes = [vp, vp, vp]
        L.grmhd_next_dt.argtypes = [vp, P(d)]
        L.grmhd_get_flags.argtypes = [vp, vp, vp]
        L.grmhd_get_geometry.argtypes = [vp, i, vp]
        L.grmhd_set_geometry.argtypes = [vp, i, vp]
        L.grmhd_fluxes_noalloc.argtypes = [P(grmhd_grid), P(grmhd_metric), P(grmhd_params), vp,
                                           vp, vp, vp]
        L.grmhd_profile.argtypes = [vp, i]
        L.grmhd_arith.argtypes = [i, vp, vp, ctypes.c_longlong, vp]
        L.grmhd_fp64_probe.argtypes = [i, i, i, ctypes.c_longlong, P(d), P(d)]
        L.grmhd_get_profile.argtypes = [vp, P(grmhd_profile_data), i]
        L.grmhd_fp64_peak.argtypes = [ctypes.c_longlong, P(d)]
        L.grmhd_batch_create.argtypes = [P(vp), i, P(vp)]
        L.grmhd_batch_destroy.argtypes = [vp]
        L.grmhd_batch_step.argtypes = [vp, i, i]
        L.grmhd_batch_get_info.argtypes = [vp, P(grmhd_batch_info)]
        L.grmhd_batch_sync.argtypes = [vp]
        L.grmhd_autotune.argtypes = [vp, i, P(d), P(d)]
        L.grmhd_set_recon_walk.argtypes = [vp, i, P(i)]
        L.grmhd_divb.argtypes = [vp, P(d), P(d)]
        L.grmhd_batch_autotune.argtypes = [vp, i, P(d), P(d)]
        L.grmhd_batch_set_launch.argtypes = [vp, i, i, i]
        L.grmhd_footprint.argtypes = [P(grmhd_grid), P(grmhd_metric), P(grmhd_params),
                                      P(ctypes.c_size_t)]
        L.grmhd_server_create.argtypes = [P(grmhd_server_config), P(vp)]
        L.grmhd_server_submit.argtypes = [vp, ctypes.c_longlong, P(grmhd_grid), P(grmhd_metric),
                                          P(grmhd_params), vp, i, vp, i, ctypes.c_longlong, d]
        L.grmhd_server_submit_electrons.argtypes = [vp, ctypes.c_longlong, P(grmhd_grid),
                                                    P(grmhd_metric), P(grmhd_params), vp, vp, i,
                                                    vp, vp, i, ctypes.c_longlong, d]
        L.grmhd_server_poll.argtypes = [vp, P(grmhd_server_result), i, i]
        L.grmhd_server_drain.argtypes = [vp, i]
        L.grmhd_server_get_stats.argtypes = [vp, P(grmhd_server_stats)]
        L.grmhd_server_now.argtypes = [vp]
        L.grmhd_server_destroy.argtypes = [vp]
        L.grmhd_decomp_create.argtypes = [P(grmhd_grid), P(grmhd_metric), P(grmhd_params),
                                          P(i), vp, P(vp)]
        L.grmhd_decomp_destroy.argtypes = [vp]
        L.grmhd_decomp_set_prims.argtypes = [vp, vp, i]
        L.grmhd_decomp_get_prims.argtypes = [vp, vp, i]
        L.grmhd_decomp_set_electrons.argtypes = [vp, vp, i]
        L.grmhd_decomp_get_electrons.argtypes = [vp, vp, i]
        L.grmhd_decomp_step.argtypes = [vp, i, P(grmhd_stats)]
        L.grmhd_decomp_get_stats.argtypes = [vp, P(grmhd_stats), i]
        L.grmhd_strerror.argtypes = [i]
        L.grmhd_strerror.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name not in ("grmhd_strerror", "grmhd_server_now"):
                getattr(L, name).restype = i
        L.grmhd_server_now.restype = d
        _lib = L
        return L


def _check(rc, where):
    if rc != GRMHD_OK:
        raise GrmhdError(rc, where)


def _ptr(a):
    """(pointer, on_device) of a C-contiguous float64 numpy array or torch
    tensor (the library reads and writes doubles)."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if a.dtype != np.float64:
            raise ValueError("array must be float64, not %s" % a.dtype)
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if str(a.dtype) != "torch.float64":
            raise ValueError("tensor must be torch.float64, not %s" % a.dtype)
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError("expected a numpy array or a torch tensor")


def fp64_peak(iters: int = 1 << 16) -> float:
    """Measured FP64 FMA throughput (FLOP/s) of the current device."""
    out = ctypes.c_double()
    _check(load().grmhd_fp64_peak(int(iters), ctypes.byref(out)), "grmhd_fp64_peak")
    return out.value


def fp64_probe(op: int = 0, chains: int = 8, blocks_per_sm: int = 8, iters: int = 1 << 14):
    """(FP64 instructions per SM per clock cycle, SM MHz measured in the
    kernel) of a loop of op (0 FMA, 1 add, 2 multiply) with `chains`
    independent chains per thread on blocks_per_sm blocks of 128 threads
    per SM."""
    r, mhz = ctypes.c_double(), ctypes.c_double()
    _check(load().grmhd_fp64_probe(int(op), int(chains), int(blocks_per_sm), int(iters),
                                   ctypes.byref(r), ctypes.byref(mhz)), "grmhd_fp64_probe")
    return r.value, mhz.value


def _structs(pr):
    g = grmhd_grid(int(pr.n[0]), int(pr.n[1]), int(pr.n[2]), pr.xmin[0], pr.xmax[0], pr.xmin[1],
                   pr.xmax[1], pr.xmin[2], pr.xmax[2])
    m = grmhd_metric(int(pr.metric), float(pr.a), float(pr.hslope))
    p = grmhd_params()
    p.gamma, p.cfl, p.t_final = float(pr.gamma), float(pr.cfl), float(pr.t_final)
    p.recon, p.floors_on = int(pr.recon), int(pr.floors)
    for d in range(3):
        for s in range(2):
            p.bc[d][s] = int(pr.bc[d][s])
    p.precision = int(getattr(pr, "precision", PREC_FP64))
    p.floor_frame = int(getattr(pr, "floor_frame", FLOOR_FLUID))
    el = getattr(pr, "electrons", None)
    if el and el["model"]:
        p.electrons = grmhd_electrons(int(el["model"]), float(el["game"]), float(el["gamp"]),
                                      float(el["fel"]), float(el["tpte_min"]), float(el["tpte_max"]))
    return g, m, p


def fluxes_noalloc(problem, P, F, stream=None):
    """Flux stage of `problem`'s grid on caller-owned device tensors, with no
    device allocation (see grmhd_fluxes_noalloc in include/grmhd.h).
    P: device [8][n3+6][n2+6][n1+6] with ghosts filled; F: device
    [3][8][n3+6][n2+6][n1+6] output.  Returns the signal-speed maxima."""
    g, m, p = _structs(problem)
    pp, pdev = _ptr(P)
    fp, fdev = _ptr(F)
    if not (pdev and fdev):
        raise ValueError("P and F must be device tensors")
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    ct = np.zeros(3)
    _check(load().grmhd_fluxes_noalloc(ctypes.byref(g), ctypes.byref(m), ctypes.byref(p), pp, fp,
                                       ct.ctypes.data, ctypes.c_void_p(stream or 0)),
           "grmhd_fluxes_noalloc")
    return ct


ARITH = {"rcp": 0, "rsqrt": 1, "sqrt": 2, "div_sigma": 3, "div_temp": 4}


def arith(fn, x, out, stream=None):
    """The step's reciprocal ("rcp"), reciprocal square root ("rsqrt"),
    square root ("sqrt") or the bounds' quotients x / 400 ("div_sigma") and
    x / 100 ("div_temp") of every element of the device tensor x into out
    (float64, same size; see grmhd_arith in include/grmhd.h)."""
    xp, xdev = _ptr(x)
    op, odev = _ptr(out)
    if not (xdev and odev):
        raise ValueError("x and out must be device tensors")
    if x.numel() != out.numel():
        raise ValueError("x and out differ in size")
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    _check(load().grmhd_arith(ARITH[fn], xp, op, int(x.numel()), ctypes.c_void_p(stream or 0)),
           "grmhd_arith")


class Sim:
    """One GRMHD simulation held on the current CUDA device.

    ``problem`` has the attributes of ``problems.Problem`` (n, xmin, xmax,
    metric, a, hslope, gamma, cfl, t_final, recon, floors, bc)."""

    def __init__(self, problem, stream=None):
        self.L = load()
        pr = problem
        self.n = tuple(int(x) for x in pr.n)
        self.s = tuple(x + 2 * NG for x in self.n)
        g, m, p = _structs(pr)
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self.h = ctypes.c_void_p()
        _check(self.L.grmhd_create(ctypes.byref(g), ctypes.byref(m), ctypes.byref(p),
                                   ctypes.c_void_p(stream or 0), ctypes.byref(self.h)),
               "grmhd_create")

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.L.grmhd_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- state ----
    def set_prims(self, P) -> None:
        n1, n2, n3 = self.n
        shape = tuple(P.shape)
        ptr, dev = _ptr(P)
        if shape == (NPRIM, n3, n2, n1):
            _check(self.L.grmhd_set_prims(self.h, ptr, dev), "grmhd_set_prims")
        elif shape == (NPRIM,) + self.s[::-1]:
            _check(self.L.grmhd_set_prims_ghost(self.h, ptr, dev), "grmhd_set_prims_ghost")
        else:
            raise ValueError("bad primitive shape %s" % (shape,))

    def set_electrons(self, K) -> None:
        """Electron entropies (kappa_tot, kappa_e), [2][n3][n2][n1] or with ghosts."""
        n1, n2, n3 = self.n
        shape = tuple(K.shape)
        if shape == (2, n3, n2, n1):
            ghosts = 0
        elif shape == (2,) + self.s[::-1]:
            ghosts = 1
        else:
            raise ValueError("bad electron shape %s" % (shape,))
        if isinstance(K, np.ndarray):
            K = np.ascontiguousarray(K, dtype=np.float64)
        ptr, dev = _ptr(K)
        _check(self.L.grmhd_set_electrons(self.h, ptr, ghosts, dev), "grmhd_set_electrons")

    def get_electrons(self, with_ghosts: bool = False):
        out = np.empty((2,) + (self.s[::-1] if with_ghosts else self.n[::-1]))
        _check(self.L.grmhd_get_electrons(self.h, out.ctypes.data, int(with_ghosts), 0),
               "grmhd_get_electrons")
        return out

    def get_prims(self, with_ghosts: bool = False, out=None):
        shape = (NPRIM,) + (self.s[::-1] if with_ghosts else self.n[::-1])
        if out is None:
            out = np.empty(shape, dtype=np.float64)
        if tuple(out.shape) != shape:
            raise ValueError("bad output shape")
        ptr, dev = _ptr(out)
        _check(self.L.grmhd_get_prims(self.h, ptr, int(with_ghosts), dev), "grmhd_get_prims")
        return out

    def step(self, nsteps: int = 1, sync: bool = True):
        if sync:
            st = grmhd_stats()
            _check(self.L.grmhd_step(self.h, int(nsteps), ctypes.byref(st)), "grmhd_step")
            return st.as_dict()
        _check(self.L.grmhd_step(self.h, int(nsteps), None), "grmhd_step")
        return None

    def stats(self):
        st = grmhd_stats()
        _check(self.L.grmhd_get_stats(self.h, ctypes.byref(st)), "grmhd_get_stats")
        return st.as_dict()

    def set_time(self, t: float, dt_prev: float, steps: int = 0) -> None:
        _check(self.L.grmhd_set_time(self.h, float(t), float(dt_prev), int(steps)), "grmhd_set_time")

    # ---- stage-level access ----
    def predictor(self) -> None:
        _check(self.L.grmhd_predictor(self.h), "grmhd_predictor")

    def fluxes(self):
        F = np.zeros((3, NPRIM) + self.s[::-1])
        ct = np.zeros(3)
        _check(self.L.grmhd_get_fluxes(self.h, F.ctypes.data, ct.ctypes.data), "grmhd_get_fluxes")
        return F, ct

    def next_dt(self) -> float:
        out = ctypes.c_double()
        _check(self.L.grmhd_next_dt(self.h, ctypes.byref(out)), "grmhd_next_dt")
        return out.value

    def flags(self):
        n1, n2, n3 = self.n
        pf = np.zeros((n3, n2, n1), dtype=np.int32)
        ff = np.zeros((n3, n2, n1), dtype=np.int32)
        _check(self.L.grmhd_get_flags(self.h, pf.ctypes.data, ff.ctypes.data), "grmhd_get_flags")
        return pf, ff

    def set_geom(self, loc: int, arr) -> None:
        """Load geometry in the layout of geom(loc) (a tabulated metric)."""
        nc = 64 if loc == 3 else 34
        a = np.ascontiguousarray(arr, dtype=np.float64)
        if a.shape != (nc, self.s[1], self.s[0]):
            raise ValueError("bad geometry shape %s" % (a.shape,))
        _check(self.L.grmhd_set_geometry(self.h, int(loc), a.ctypes.data), "grmhd_set_geometry")

    def profile(self, enable: bool = True) -> None:
        _check(self.L.grmhd_profile(self.h, int(enable)), "grmhd_profile")

    def get_profile(self, reset: bool = False):
        """{class: (ms, launches)} since the last reset."""
        pd = grmhd_profile_data()
        _check(self.L.grmhd_get_profile(self.h, ctypes.byref(pd), int(reset)), "grmhd_get_profile")
        return {c: (pd.ms[q], pd.launches[q]) for q, c in enumerate(KCLASSES)}

    def divb(self):
        """(max |corner div sqrt(-g) B|, max |sqrt(-g) B^d|) of the state."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(self.L.grmhd_divb(self.h, ctypes.byref(a), ctypes.byref(b)), "grmhd_divb")
        return a.value, b.value

    def autotune(self, trials: int = 3):
        """Pick the block sizes of the step's heavy kernels by timing;
        returns (ms before, ms after) for one pass of them."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(self.L.grmhd_autotune(self.h, int(trials), ctypes.byref(a), ctypes.byref(b)),
               "grmhd_autotune")
        return a.value, b.value

    def set_recon_walk(self, zones_per_thread: int = 0) -> int:
        """Zones per thread of the FP64 reconstruction (1, 2, 4, 8, 16; 0:
        automatic); returns the length in use.  Values do not depend on it."""
        c = ctypes.c_int()
        _check(self.L.grmhd_set_recon_walk(self.h, int(zones_per_thread), ctypes.byref(c)),
               "grmhd_set_recon_walk")
        return c.value

    def geom(self, loc: int) -> np.ndarray:
        nc = 64 if loc == 3 else 34
        out = np.zeros((nc, self.s[1], self.s[0]))
        _check(self.L.grmhd_get_geometry(self.h, int(loc), out.ctypes.data), "grmhd_get_geometry")
        return out


class Batch:
    """Several simulations advanced together by one set of launches per
    step (``grmhd_batch_*``).  The batch references the ``Sim`` objects and
    keeps them alive; each grid's result is bitwise its result alone."""

    def __init__(self, sims):
        self.L = load()
        self.sims = list(sims)
        arr = (ctypes.c_void_p * len(self.sims))(*[s.h.value for s in self.sims])
        self.h = ctypes.c_void_p()
        _check(self.L.grmhd_batch_create(arr, len(self.sims), ctypes.byref(self.h)),
               "grmhd_batch_create")

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.L.grmhd_batch_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def step(self, nsteps: int = 1, graph: bool = True, sync: bool = False) -> None:
        _check(self.L.grmhd_batch_step(self.h, int(nsteps), int(graph)), "grmhd_batch_step")
        if sync:
            self.sync()

    def sync(self) -> None:
        _check(self.L.grmhd_batch_sync(self.h), "grmhd_batch_sync")

    def autotune(self, trials: int = 3):
        """Pick block sizes and block orders of the heavy kernels by timing;
        returns (ms before, ms after) for one pass of them."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(self.L.grmhd_batch_autotune(self.h, int(trials), ctypes.byref(a), ctypes.byref(b)),
               "grmhd_batch_autotune")
        return a.value, b.value

    def set_launch(self, kclass: str, threads: int, order: int) -> None:
        """Fix threads per block and block order (0 batch order, 1 largest
        grid first, 2 round robin) of the "recon", "flux" or "update" kernels."""
        _check(self.L.grmhd_batch_set_launch(self.h, KCLASSES.index(kclass), int(threads), int(order)),
               "grmhd_batch_set_launch")

    def info(self):
        out = grmhd_batch_info()
        _check(self.L.grmhd_batch_get_info(self.h, ctypes.byref(out)), "grmhd_batch_get_info")
        return out.as_dict()


def footprint(problem) -> int:
    """Device bytes a simulation of this problem holds."""
    g, m, p = _structs(problem)
    out = ctypes.c_size_t()
    _check(load().grmhd_footprint(ctypes.byref(g), ctypes.byref(m), ctypes.byref(p), ctypes.byref(out)),
           "grmhd_footprint")
    return out.value


class Server:
    """The serving request loop (``grmhd_server_*``): submit simulations as
    they arrive, poll finished results.  Input and output arrays are kept
    referenced here until their result has been polled."""

    FIFO, SWF = 0, 1  # admission: arrival order / smallest work first

    def __init__(self, hbm_budget: int = 0, max_active_zones: int = 0, quantum: int = 8,
                 use_graph: bool = True, policy: int = 0):
        self.L = load()
        cfg = grmhd_server_config(int(hbm_budget), int(max_active_zones), int(quantum), int(use_graph),
                                  int(policy))
        self.h = ctypes.c_void_p()
        _check(self.L.grmhd_server_create(ctypes.byref(cfg), ctypes.byref(self.h)), "grmhd_server_create")
        self._held = {}

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.L.grmhd_server_destroy(self.h)
            self.h = ctypes.c_void_p()
            self._held = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def now(self) -> float:
        return self.L.grmhd_server_now(self.h)

    def submit(self, rid: int, problem, nsteps: int, t_arrival: float = -1.0,
               out_ghosts: bool = False) -> np.ndarray:
        """Queue a simulation of ``problem`` for ``nsteps`` cycles; returns the
        host array its result will be written to.  A problem with fixed
        boundary ghosts (``info['P_ghost']``) is submitted with its ghosts."""
        g, m, p = _structs(problem)
        Pg = problem.info.get("P_ghost") if problem.info else None
        P_in = np.ascontiguousarray(Pg if Pg is not None else problem.P, dtype=np.float64)
        n1, n2, n3 = (int(x) for x in problem.n)
        shape = (NPRIM, n3 + 2 * NG, n2 + 2 * NG, n1 + 2 * NG) if out_ghosts else (NPRIM, n3, n2, n1)
        out = np.empty(shape, dtype=np.float64)
        el = getattr(problem, "electrons", None)
        if el and el["model"]:  # the electron entropies travel with the request
            Kg = problem.info.get("K_ghost") if problem.info else None
            K_in = np.ascontiguousarray(Kg if Pg is not None else problem.K, dtype=np.float64)
            K_out = np.empty((2,) + shape[1:], dtype=np.float64)
            _check(self.L.grmhd_server_submit_electrons(
                self.h, int(rid), ctypes.byref(g), ctypes.byref(m), ctypes.byref(p),
                P_in.ctypes.data, K_in.ctypes.data, int(Pg is not None), out.ctypes.data,
                K_out.ctypes.data, int(out_ghosts), int(nsteps), float(t_arrival)),
                "grmhd_server_submit_electrons")
            self._held[int(rid)] = (P_in, out, K_in, K_out)
        else:
            _check(self.L.grmhd_server_submit(self.h, int(rid), ctypes.byref(g), ctypes.byref(m),
                                              ctypes.byref(p), P_in.ctypes.data, int(Pg is not None),
                                              out.ctypes.data, int(out_ghosts), int(nsteps),
                                              float(t_arrival)), "grmhd_server_submit")
            self._held[int(rid)] = (P_in, out)
        return out

    def poll(self, max_results: int = 64, wait_ms: int = 0):
        """Finished requests as dicts (id, status, zones, steps, t_arrival,
        t_admit, t_done, stats, P)."""
        buf = (grmhd_server_result * max(int(max_results), 1))()
        n = self.L.grmhd_server_poll(self.h, buf, int(max_results), int(wait_ms))
        if n < 0:
            raise GrmhdError(n, "grmhd_server_poll")
        out = []
        for q in range(n):
            r = buf[q]
            held = self._held.pop(int(r.id), (None, None))
            out.append({"id": r.id, "status": r.status, "zones": r.zones, "steps": r.steps,
                        "t_arrival": r.t_arrival, "t_admit": r.t_admit, "t_done": r.t_done,
                        "stats": r.stats.as_dict(), "P": held[1],
                        "K": held[3] if len(held) > 3 else None})
        return out

    def drain(self, timeout_ms: int = -1) -> None:
        _check(self.L.grmhd_server_drain(self.h, int(timeout_ms)), "grmhd_server_drain")

    def stats(self):
        out = grmhd_server_stats()
        _check(self.L.grmhd_server_get_stats(self.h, ctypes.byref(out)), "grmhd_server_get_stats")
        return out.as_dict()


class Decomp:
    """One grid split into nblocks[0] x nblocks[1] x nblocks[2] blocks
    (``grmhd_decomp_*``); bitwise the same evolution as ``Sim``."""

    def __init__(self, problem, nblocks, stream=None):
        self.L = load()
        self.n = tuple(int(x) for x in problem.n)
        self.s = tuple(x + 2 * NG for x in self.n)
        g, m, p = _structs(problem)
        nb = (ctypes.c_int * 3)(*[int(x) for x in nblocks])
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self.h = ctypes.c_void_p()
        _check(self.L.grmhd_decomp_create(ctypes.byref(g), ctypes.byref(m), ctypes.byref(p), nb,
                                          ctypes.c_void_p(stream or 0), ctypes.byref(self.h)),
               "grmhd_decomp_create")

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.L.grmhd_decomp_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_prims(self, P) -> None:
        a = np.ascontiguousarray(P, dtype=np.float64)
        n1, n2, n3 = self.n
        if a.shape == (NPRIM, n3, n2, n1):
            ghosts = 0
        elif a.shape == (NPRIM,) + self.s[::-1]:
            ghosts = 1
        else:
            raise ValueError("bad primitive shape %s" % (a.shape,))
        _check(self.L.grmhd_decomp_set_prims(self.h, a.ctypes.data, ghosts), "grmhd_decomp_set_prims")

    def get_prims(self, with_ghosts: bool = False) -> np.ndarray:
        out = np.zeros((NPRIM,) + (self.s[::-1] if with_ghosts else self.n[::-1]))
        _check(self.L.grmhd_decomp_get_prims(self.h, out.ctypes.data, int(with_ghosts)),
               "grmhd_decomp_get_prims")
        return out

    def set_electrons(self, K) -> None:
        a = np.ascontiguousarray(K, dtype=np.float64)
        n1, n2, n3 = self.n
        if a.shape == (2, n3, n2, n1):
            ghosts = 0
        elif a.shape == (2,) + self.s[::-1]:
            ghosts = 1
        else:
            raise ValueError("bad electron shape %s" % (a.shape,))
        _check(self.L.grmhd_decomp_set_electrons(self.h, a.ctypes.data, ghosts),
               "grmhd_decomp_set_electrons")

    def get_electrons(self, with_ghosts: bool = False) -> np.ndarray:
        out = np.zeros((2,) + (self.s[::-1] if with_ghosts else self.n[::-1]))
        _check(self.L.grmhd_decomp_get_electrons(self.h, out.ctypes.data, int(with_ghosts)),
               "grmhd_decomp_get_electrons")
        return out

    def step(self, nsteps: int = 1):
        st = grmhd_stats()
        _check(self.L.grmhd_decomp_step(self.h, int(nsteps), ctypes.byref(st)), "grmhd_decomp_step")
        return st.as_dict()

    def stats(self, check: bool = False):
        st = grmhd_stats()
        _check(self.L.grmhd_decomp_get_stats(self.h, ctypes.byref(st), int(check)),
               "grmhd_decomp_get_stats")
        return st.as_dict()
