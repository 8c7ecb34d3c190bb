"""ctypes binding of the FP64 CPU oracle (oracle/grmhd_oracle.cpp).

TEST INFRASTRUCTURE ONLY: the oracle is the correctness reference of the
CUDA library.  Only tests/, ``__graft_entry__.smoke()`` and bench.py's
oracle leg (the CPU baseline, ``--impl reference`` and the accuracy figures
measured against the oracle) may import it.  It shares no code
with ``paper_2110_10191_gb300`` and imports nothing from it.

``build()`` compiles two shared objects with g++ (no -march flags, so the
same source builds on x86_64 and aarch64):

* ``liboracle.so``        -- real == double, -ffp-contract=off
* ``liboracle_count.so``  -- the same source with a counting scalar type that
  tallies add/sub, mul, div and sqrt of the step (algorithmic FP64 work).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "grmhd_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict = {}

NPRIM = 8
NG = 3
# floor flag bits (as in grmhd_oracle.cpp)
FF_GAMMA, FF_RHO_GEOM, FF_U_GEOM, FF_SIGMA, FF_BETA, FF_TEMP = 1, 2, 4, 8, 16, 32
FF_DRIFT, FF_DRIFT_FAIL, FF_KTOT = 64, 128, 256
# electron heating models
ELEC_OFF, ELEC_CONSTANT, ELEC_KAWAZURA, ELEC_WERNER, ELEC_ROWAN, ELEC_SHARMA, ELEC_HOWES = range(7)
METRIC_MINKOWSKI, METRIC_MKS_KERR = 0, 1
BC_PERIODIC, BC_OUTFLOW, BC_POLAR, BC_FIXED = 0, 1, 2, 3
RECON_MC, RECON_WENO5 = 0, 1


def _lib_path(counting: bool) -> str:
    return os.path.join(_BUILD, "liboracle_count.so" if counting else "liboracle.so")


def build(force: bool = False) -> None:
    """Compile both oracle builds (g++ -O2 -ffp-contract=off)."""
    os.makedirs(_BUILD, exist_ok=True)
    jobs = []
    for counting in (False, True):
        out = _lib_path(counting)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", out + ".tmp", _SRC]
        if counting:
            cmd.insert(1, "-DORACLE_COUNT")
        jobs.append((subprocess.Popen(cmd), out))
    for p, out in jobs:
        if p.wait() != 0:
            raise RuntimeError("oracle build failed: %s" % out)
        os.replace(out + ".tmp", out)


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def lib(counting: bool = False) -> ctypes.CDLL:
    """The oracle library.  ORACLE_LIB, when set, names another build of the
    plain (non-counting) oracle to load instead: the mutation tests point it
    at copies of the source with a planted mistake."""
    with _LOCK:
        if counting in _LIBS:
            return _LIBS[counting]
        path = os.environ.get("ORACLE_LIB") if not counting else None
        if not path:
            path = _lib_path(counting)
            if not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
                build()
        L = ctypes.CDLL(path)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        P = ctypes.POINTER
        L.oracle_create.restype = vp
        L.oracle_create.argtypes = [P(i), P(d), P(d), i, d, d, d, d, d, i, i, P(i)]
        L.oracle_destroy.argtypes = [vp]
        L.oracle_set_prims.argtypes = [vp, P(d)]
        L.oracle_set_prims_ghost.argtypes = [vp, P(d)]
        L.oracle_get_prims.argtypes = [vp, P(d), i]
        L.oracle_step.argtypes = [vp, i]
        L.oracle_step.restype = i
        L.oracle_get_time.argtypes = [vp, P(d)]
        L.oracle_set_time.argtypes = [vp, d, d, ctypes.c_long]
        L.oracle_predictor.argtypes = [vp]
        L.oracle_predictor.restype = i
        L.oracle_get_counters.argtypes = [vp, P(ctypes.c_long)]
        L.oracle_get_flags.argtypes = [vp, P(i), P(i)]
        L.oracle_get_fluxes.argtypes = [vp, P(d), P(d)]
        L.oracle_next_dt.argtypes = [vp]
        L.oracle_next_dt.restype = d
        L.oracle_get_geom.argtypes = [vp, i, P(d)]
        L.oracle_geom_at.argtypes = [i, d, d, P(d), P(d)]
        L.oracle_prim_to_flux.argtypes = [i, d, d, P(d), d, P(d), i, P(d)]
        L.oracle_state_at.argtypes = [i, d, d, P(d), P(d), P(d)]
        L.oracle_cons_to_prim.argtypes = [i, d, d, P(d), d, P(d), P(d), P(d)]
        L.oracle_cons_to_prim.restype = i
        L.oracle_vchar.argtypes = [i, d, d, P(d), d, P(d), i, P(d)]
        L.oracle_source_at.argtypes = [i, d, d, P(d), d, P(d), P(d)]
        L.oracle_floors_at.argtypes = [i, d, d, P(d), d, P(d)]
        L.oracle_floors_at.restype = i
        L.oracle_floors_drift_at.argtypes = [i, d, d, P(d), d, P(d), P(d)]
        L.oracle_floors_drift_at.restype = i
        L.oracle_set_floor_frame.argtypes = [vp, i]
        L.oracle_set_electrons.argtypes = [vp, i, d, d, d, d, d]
        L.oracle_set_K.argtypes = [vp, P(d), i]
        L.oracle_get_K.argtypes = [vp, P(d), i]
        L.oracle_elec_fraction.argtypes = [i, d, d, d, d, d, d, d, d]
        L.oracle_elec_fraction.restype = d
        L.oracle_elec_heat.argtypes = [d, d, d, d, d, d, d]
        L.oracle_elec_heat.restype = d
        L.oracle_recon.argtypes = [i, P(d), P(d)]
        L.oracle_recon_faces.argtypes = [P(d), P(d)]
        L.oracle_op_counts.argtypes = [P(d), i]
        L.oracle_is_counting.restype = i
        _LIBS[counting] = L
        return L


class Oracle:
    """One simulation held by the oracle.

    ``problem`` is a :class:`paper_2110_10191_gb300.problems.Problem` (or any
    object with the same attributes: n, xmin, xmax, metric, a, hslope, gamma,
    cfl, t_final, recon, floors, bc)."""

    def __init__(self, problem, counting: bool = False):
        self.L = lib(counting)
        pr = problem
        self.n = tuple(int(x) for x in pr.n)
        self.s = tuple(x + 2 * NG for x in self.n)
        n = np.array(self.n, dtype=np.int32)
        xmin = np.array(pr.xmin, dtype=np.float64)
        xmax = np.array(pr.xmax, dtype=np.float64)
        bc = np.array(pr.bc, dtype=np.int32).reshape(6)
        self.h = self.L.oracle_create(_ip(n), _dp(xmin), _dp(xmax), int(pr.metric), float(pr.a),
                                      float(pr.hslope), float(pr.gamma), float(pr.cfl),
                                      float(pr.t_final), int(pr.recon), int(pr.floors), _ip(bc))
        self.L.oracle_set_floor_frame(self.h, int(getattr(pr, "floor_frame", 0)))
        el = getattr(pr, "electrons", None)
        self.electrons = bool(el and el["model"])
        if self.electrons:
            self.L.oracle_set_electrons(self.h, int(el["model"]), float(el["game"]),
                                        float(el["gamp"]), float(el["fel"]),
                                        float(el["tpte_min"]), float(el["tpte_max"]))

    def set_K(self, K) -> None:
        """Electron entropies (kappa_tot, kappa_e): [2][n3][n2][n1] or with ghosts."""
        K = np.ascontiguousarray(K, dtype=np.float64)
        ghosts = 1 if K.shape == (2,) + self.s[::-1] else 0
        if not ghosts and K.shape != (2,) + self.n[::-1]:
            raise ValueError("bad electron shape %s" % (K.shape,))
        self.L.oracle_set_K(self.h, _dp(K), ghosts)

    def get_K(self, with_ghosts: bool = False) -> np.ndarray:
        out = np.zeros((2,) + (self.s[::-1] if with_ghosts else self.n[::-1]))
        self.L.oracle_get_K(self.h, _dp(out), int(with_ghosts))
        return out

    def close(self):
        if self.h:
            self.L.oracle_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_prims(self, P: np.ndarray) -> None:
        P = np.ascontiguousarray(P, dtype=np.float64)
        n1, n2, n3 = self.n
        if P.shape == (NPRIM, n3, n2, n1):
            self.L.oracle_set_prims(self.h, _dp(P))
        elif P.shape == (NPRIM,) + self.s[::-1]:
            self.L.oracle_set_prims_ghost(self.h, _dp(P))
        else:
            raise ValueError("bad primitive shape %s" % (P.shape,))

    def get_prims(self, with_ghosts: bool = False) -> np.ndarray:
        shape = (NPRIM,) + (self.s[::-1] if with_ghosts else self.n[::-1])
        out = np.empty(shape, dtype=np.float64)
        self.L.oracle_get_prims(self.h, _dp(out), int(with_ghosts))
        return out

    def step(self, nsteps: int = 1) -> int:
        return int(self.L.oracle_step(self.h, int(nsteps)))

    def set_time(self, t: float, dt_prev: float, nstep: int = 0) -> None:
        self.L.oracle_set_time(self.h, float(t), float(dt_prev), int(nstep))

    def predictor(self) -> int:
        """Predictor stage only: P <- P^{n+1/2}; t is not advanced."""
        return int(self.L.oracle_predictor(self.h))

    def time(self):
        out = np.zeros(3)
        self.L.oracle_get_time(self.h, _dp(out))
        return float(out[0]), float(out[1]), int(out[2])

    def counters(self):
        out = np.zeros(3, dtype=np.int64)
        self.L.oracle_get_counters(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_long)))
        return {"inv_failures": int(out[0]), "floor_hits": int(out[1]),
                "unrecoverable": int(out[2])}

    def flags(self):
        n1, n2, n3 = self.n
        pf = np.zeros((n3, n2, n1), dtype=np.int32)
        ff = np.zeros((n3, n2, n1), dtype=np.int32)
        self.L.oracle_get_flags(self.h, _ip(pf), _ip(ff))
        return pf, ff

    def fluxes(self):
        F = np.zeros((3, NPRIM) + self.s[::-1])
        ct = np.zeros(3)
        self.L.oracle_get_fluxes(self.h, _dp(F), _dp(ct))
        return F, ct

    def next_dt(self) -> float:
        return float(self.L.oracle_next_dt(self.h))

    def geom(self, loc: int) -> np.ndarray:
        nc = 64 if loc == 3 else 34
        out = np.zeros((nc, self.s[1], self.s[0]))
        self.L.oracle_get_geom(self.h, int(loc), _dp(out))
        return out


# ---------------------------------------------------------------- pointwise

def _X(X):
    X = np.zeros(4) + np.asarray(X, dtype=np.float64)
    return np.ascontiguousarray(X)


def geom_at(kind, a, h, X):
    """dict with gcov (4x4), gcon (4x4), gdet, alpha, conn (4x4x4) at X."""
    out = np.zeros(98)
    lib().oracle_geom_at(int(kind), float(a), float(h), _dp(_X(X)), _dp(out))
    return {"gcov": out[:16].reshape(4, 4).copy(), "gcon": out[16:32].reshape(4, 4).copy(),
            "gdet": float(out[32]), "alpha": float(out[33]),
            "conn": out[34:98].reshape(4, 4, 4).copy()}


def prim_to_flux(kind, a, h, X, gam, P, dir):
    P = np.ascontiguousarray(P, dtype=np.float64)
    F = np.zeros(NPRIM)
    lib().oracle_prim_to_flux(int(kind), float(a), float(h), _dp(_X(X)), float(gam), _dp(P),
                              int(dir), _dp(F))
    return F


def state_at(kind, a, h, X, P):
    P = np.ascontiguousarray(P, dtype=np.float64)
    out = np.zeros(9)
    lib().oracle_state_at(int(kind), float(a), float(h), _dp(_X(X)), _dp(P), _dp(out))
    return {"bsq": float(out[0]), "ucon": out[1:5].copy(), "bcon": out[5:9].copy()}


def cons_to_prim(kind, a, h, X, gam, U, Pguess):
    U = np.ascontiguousarray(U, dtype=np.float64)
    Pg = np.ascontiguousarray(Pguess, dtype=np.float64)
    P = np.zeros(NPRIM)
    rc = lib().oracle_cons_to_prim(int(kind), float(a), float(h), _dp(_X(X)), float(gam),
                                   _dp(U), _dp(Pg), _dp(P))
    return int(rc), P


def vchar(kind, a, h, X, gam, P, dir):
    P = np.ascontiguousarray(P, dtype=np.float64)
    out = np.zeros(2)
    lib().oracle_vchar(int(kind), float(a), float(h), _dp(_X(X)), float(gam), _dp(P), int(dir),
                       _dp(out))
    return float(out[0]), float(out[1])


def source_at(kind, a, h, X, gam, P):
    P = np.ascontiguousarray(P, dtype=np.float64)
    out = np.zeros(NPRIM)
    lib().oracle_source_at(int(kind), float(a), float(h), _dp(_X(X)), float(gam), _dp(P),
                           _dp(out))
    return out


def floors_at(kind, a, h, X, gam, P):
    P = np.array(P, dtype=np.float64)
    fl = lib().oracle_floors_at(int(kind), float(a), float(h), _dp(_X(X)), float(gam), _dp(P))
    return int(fl), P


def elec_fraction(model, gam, game, gamp, fel, rho, u, kel, bsq):
    """Electron heating fraction of one zone (model as ELEC_* of the oracle)."""
    return lib().oracle_elec_fraction(int(model), float(gam), float(game), float(gamp), float(fel),
                                      float(rho), float(u), float(kel), float(bsq))


def elec_heat(gam, game, rho_s, fel, ktot_new, ktot_adv, kel_adv):
    """One heating update of kappa_e."""
    return lib().oracle_elec_heat(float(gam), float(game), float(rho_s), float(fel),
                                  float(ktot_new), float(ktot_adv), float(kel_adv))


def floors_drift_at(kind, a, h, X, gam, P):
    """Drift-frame bounds at one point: (flags, bounded P, P before the
    closing fluid-frame pass or None when no parcel was added)."""
    P = np.array(P, dtype=np.float64)
    pre = np.zeros(8)
    fl = lib().oracle_floors_drift_at(int(kind), float(a), float(h), _dp(_X(X)), float(gam),
                                      _dp(P), _dp(pre))
    return int(fl), P, (pre if fl & FF_DRIFT else None)


def recon(kind, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(2)
    lib().oracle_recon(int(kind), _dp(x), _dp(out))
    return float(out[0]), float(out[1])


def recon_faces(x):
    """WENO5 (low, high) face values of the middle zone, each face from its
    own smoothness indicators (the single-face form)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(2)
    lib().oracle_recon_faces(_dp(x), _dp(out))
    return out


PHASES = ["flux", "ct", "update", "fixup", "other", "recon"]


def op_counts(reset: bool = False):
    """Counting build: {phase: {add, mul, div, sqrt}} since the last reset
    (flux: face fluxes from the reconstructed states; recon: reconstruction)."""
    out = np.zeros(24)
    lib(True).oracle_op_counts(_dp(out), int(reset))
    return {ph: {"add": out[4 * q], "mul": out[4 * q + 1], "div": out[4 * q + 2],
                 "sqrt": out[4 * q + 3]} for q, ph in enumerate(PHASES)}
