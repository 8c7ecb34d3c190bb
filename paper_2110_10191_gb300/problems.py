"""Seeded, synthetic initial conditions for the GRMHD step.

This module is the one input producer that both the CUDA library's tests and
the oracle's tests use.  It holds none of the step's arithmetic: it builds a
grid description and a primitive array ``P[8][n3][n2][n1]`` (rho, u,
utilde^1..3, B^1..3) from closed-form problem definitions, with its own
numpy metric code for the set-up.

Problems (all with GM = c = 1, the paper's units, "Implementation Notes"):

* ``linear_mode``  -- flat-space linear MHD eigenmode (the paper's linear-mode
  convergence test, "Tests" section).  The eigenvector is the numpy/LAPACK
  eigendecomposition of the special-relativistic MHD flux Jacobian along k,
  the Jacobians taken by complex-step differentiation of the continuum
  conserved variables and fluxes (written here, in numpy, for set-up only).
* ``fm_torus``     -- Fishbone-Moncrief (1976) torus around a Kerr black hole
  in modified Kerr-Schild coordinates (the paper's scaling workload, "Scaling"
  section), density normalised to max rho = 1 ("Implementation Notes"),
  poloidal field from A_phi ~ max(rho/rho_max - 0.2, 0) normalised to a
  gas-to-magnetic pressure ratio, seeded perturbation of u.
* ``orszag_tang``  -- flat periodic Orszag-Tang vortex (batched workloads).
* ``batch_2d``     -- many uneven flat 2D grids of modes and vortices (batched
  workload).
* ``serving_stream`` -- Poisson arrivals of tori and Bondi inflows of random
  size, length and precision (serving workload).

Random numbers come from a counter-based generator (splitmix64 of
seed and zone index), so a zone's value does not depend on the grid split.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional

import numpy as np

NPRIM = 8
RHO, UU, U1, U2, U3, B1, B2, B3 = range(8)
METRIC_MINKOWSKI, METRIC_MKS_KERR = 0, 1
BC_PERIODIC, BC_OUTFLOW, BC_POLAR, BC_FIXED = 0, 1, 2, 3
RECON_MC, RECON_WENO5 = 0, 1


@dataclasses.dataclass
class Problem:
    """Grid, metric, parameters and interior primitives of one simulation."""
    name: str
    n: tuple                     # (n1, n2, n3) interior zones
    xmin: tuple
    xmax: tuple
    metric: int
    a: float
    hslope: float
    gamma: float
    cfl: float
    t_final: float
    recon: int
    floors: int
    bc: tuple                    # ((x1 lo, x1 hi), (x2 lo, x2 hi), (x3 lo, x3 hi))
    P: np.ndarray                # [8][n3][n2][n1] float64
    info: dict = dataclasses.field(default_factory=dict)
    precision: int = 0           # 0 FP64, 1 mixed (FP32 reconstruction and fluxes)
    floor_frame: int = 0         # bounds: 0 fluid frame, 1 drift frame
    # electron entropies: model and constants (None: not evolved), and the
    # initial (kappa_tot, kappa_e) as [2][n3][n2][n1]
    electrons: Optional[dict] = None
    K: Optional[np.ndarray] = None
    exact: Optional[Callable[[float], np.ndarray]] = None

    @property
    def zones(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])


# electron heating models (the five of the paper's list, and a constant share)
ELEC_OFF, ELEC_CONSTANT, ELEC_KAWAZURA, ELEC_WERNER, ELEC_ROWAN, ELEC_SHARMA, ELEC_HOWES = range(7)


def with_electrons(pr, model, game=4.0 / 3.0, gamp=5.0 / 3.0, fel=0.5, tpte_min=1e-3,
                   tpte_max=1e3, ue_frac=0.1, K=None):
    """A copy of `pr` that evolves the electron entropies.  Initial data:
    kappa_tot = (gamma - 1) u / rho^gamma and electrons holding the fraction
    ue_frac of the internal energy, kappa_e = (gamma_e - 1) ue_frac u /
    rho^gamma_e (or K as given).  Problems with FIXED ghosts get the same
    recipe on their ghost zones (info["K_ghost"])."""
    def kappa(P):
        rho, u = P[0], P[1]
        return np.stack([(pr.gamma - 1.0) * u / rho ** pr.gamma,
                         (game - 1.0) * ue_frac * u / rho ** game])
    info = dict(pr.info)
    Pg = info.get("P_ghost")
    if Pg is not None:
        with np.errstate(divide="ignore", invalid="ignore"):
            Kg = np.nan_to_num(kappa(Pg))
        info["K_ghost"] = Kg
    el = dict(model=int(model), game=float(game), gamp=float(gamp), fel=float(fel),
              tpte_min=float(tpte_min), tpte_max=float(tpte_max))
    return dataclasses.replace(pr, electrons=el, K=kappa(pr.P) if K is None else K, info=info)


# --------------------------------------------------------------------------
# counter-based uniform random numbers
# --------------------------------------------------------------------------

def splitmix_uniform(seed: int, index: np.ndarray) -> np.ndarray:
    """U[0,1) from the splitmix64 finaliser of (seed << 32) ^ index."""
    with np.errstate(over="ignore"):
        z = (np.uint64(seed) << np.uint64(32)) ^ index.astype(np.uint64)
        z = z + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# --------------------------------------------------------------------------
# flat-space linear modes
# --------------------------------------------------------------------------

def _srmhd_U_F(P, gam):
    """Continuum conserved variables and x/y fluxes of special-relativistic
    ideal MHD in Cartesian coordinates (complex-safe, for complex-step
    Jacobians).  Same conventions as the step: U = (rho u^t, T^t_t + rho u^t,
    T^t_i, B^i)."""
    rho, u = P[0], P[1]
    ut = P[2:5]
    B = P[5:8]
    gamma = np.sqrt(1.0 + ut[0] ** 2 + ut[1] ** 2 + ut[2] ** 2)
    ucon = np.array([gamma, ut[0], ut[1], ut[2]])
    ucov = np.array([-gamma, ut[0], ut[1], ut[2]])
    bt = B[0] * ucov[1] + B[1] * ucov[2] + B[2] * ucov[3]
    bcon = np.array([bt, (B[0] + bt * ucon[1]) / gamma, (B[1] + bt * ucon[2]) / gamma,
                     (B[2] + bt * ucon[3]) / gamma])
    bcov = np.array([-bcon[0], bcon[1], bcon[2], bcon[3]])
    bsq = bcon[0] * bcov[0] + bcon[1] * bcov[1] + bcon[2] * bcov[2] + bcon[3] * bcov[3]
    p = (gam - 1.0) * u
    w = rho + u + p + bsq
    pt = p + 0.5 * bsq

    def row(mu):
        T = np.array([w * ucon[mu] * ucov[nu] - bcon[mu] * bcov[nu] for nu in range(4)])
        T[mu] = T[mu] + pt
        F = np.zeros(8, dtype=T.dtype)
        F[0] = rho * ucon[mu]
        F[1] = T[0] + F[0]
        F[2:5] = T[1:4]
        for j in range(3):
            F[5 + j] = bcon[j + 1] * ucon[mu] - bcon[mu] * ucon[j + 1]
        return F

    return row(0), row(1), row(2)


def srmhd_jacobians(P0, gam, h=1e-30):
    """dU/dP, dF1/dP, dF2/dP at P0 by complex-step differentiation."""
    J = [np.zeros((8, 8)) for _ in range(3)]
    for j in range(8):
        Pc = np.array(P0, dtype=np.complex128)
        Pc[j] += 1j * h
        outs = _srmhd_U_F(Pc, gam)
        for m in range(3):
            J[m][:, j] = outs[m].imag / h
    return J


def mode_eigensystem(P0, gam, khat):
    """Eigen-speeds (ascending) and real eigenvectors of the linearised
    system along khat: (dU/dP)^-1 (khat_x dF1/dP + khat_y dF2/dP)."""
    JU, J1, J2 = srmhd_jacobians(P0, gam)
    A = np.linalg.solve(JU, khat[0] * J1 + khat[1] * J2)
    lam, vec = np.linalg.eig(A)
    order = np.argsort(lam.real)
    lam = lam.real[order]
    vec = vec[:, order]
    out = []
    for q in range(8):
        v = vec[:, q]
        m = np.argmax(np.abs(v))
        v = (v / v[m]).real
        out.append(v / np.max(np.abs(v)))
    return lam, np.array(out).T


def linear_mode(n: int = 64, kind: str = "fast", amp: float = 1e-4, gamma: float = 4.0 / 3.0,
                kvec=(2 * math.pi, 2 * math.pi), rho0: float = 1.0, u0: float = 1.0,
                B0=(1.0, 0.0, 0.0), cfl: float = 0.9, recon: int = RECON_MC,
                periods: float = 1.0, n2: Optional[int] = None) -> Problem:
    """A flat 2D linear eigenmode on [0,1]^2, n x n2 x 1 zones, periodic."""
    n1 = int(n)
    n2 = int(n if n2 is None else n2)
    P0 = np.array([rho0, u0, 0.0, 0.0, 0.0, B0[0], B0[1], B0[2]])
    kx, ky = float(kvec[0]), float(kvec[1])
    kmag = math.hypot(kx, ky)
    khat = np.array([kx / kmag, ky / kmag])
    lam, vec = mode_eigensystem(P0, gamma, khat)
    # positive speeds, ascending: slow < alfven < fast (zero modes excluded)
    pos = [q for q in range(8) if lam[q] > 1e-10]
    idx = {"slow": pos[0], "alfven": pos[1], "fast": pos[-1]}[kind]
    speed = float(lam[idx])
    dP = vec[:, idx].copy()
    omega = speed * kmag
    period = 2.0 * math.pi / omega
    x1 = (np.arange(n1) + 0.5) / n1
    x2 = (np.arange(n2) + 0.5) / n2
    X, Y = np.meshgrid(x1, x2, indexing="xy")  # [n2][n1]

    def exact(t: float) -> np.ndarray:
        ph = np.cos(kx * X + ky * Y - omega * t)
        P = np.empty((NPRIM, 1, n2, n1))
        for v in range(NPRIM):
            P[v, 0] = P0[v] + amp * dP[v] * ph
        return P

    return Problem(
        name="linear_mode_%s_%dx%d" % (kind, n1, n2), n=(n1, n2, 1), xmin=(0.0, 0.0, 0.0),
        xmax=(1.0, 1.0, 1.0), metric=METRIC_MINKOWSKI, a=0.0, hslope=1.0, gamma=gamma, cfl=cfl,
        t_final=periods * period, recon=recon, floors=0,
        bc=((BC_PERIODIC,) * 2,) * 3, P=exact(0.0),
        info={"speed": speed, "omega": omega, "period": period, "dP": dP, "P0": P0,
              "amp": amp, "k": (kx, ky), "eigenvalues": lam},
        exact=exact)


# --------------------------------------------------------------------------
# Orszag-Tang vortex
# --------------------------------------------------------------------------

def orszag_tang(n: int = 128, scale: float = 1.0, gamma: float = 5.0 / 3.0, cfl: float = 0.9,
                recon: int = RECON_MC, t_final: float = 0.0) -> Problem:
    """Flat periodic [0,1]^2: rho = 25/9, p = 5/3, utilde = 0.5(-sin 2pi y,
    sin 2pi x), B = s(-sin 2pi y, sin 4pi x)."""
    x1 = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x1, x1, indexing="xy")
    P = np.zeros((NPRIM, 1, n, n))
    P[RHO, 0] = 25.0 / 9.0
    P[UU, 0] = (5.0 / 3.0) / (gamma - 1.0)
    P[U1, 0] = -0.5 * np.sin(2 * math.pi * Y)
    P[U2, 0] = 0.5 * np.sin(2 * math.pi * X)
    P[B1, 0] = -scale * np.sin(2 * math.pi * Y)
    P[B2, 0] = scale * np.sin(4 * math.pi * X)
    return Problem(name="orszag_tang_%d" % n, n=(n, n, 1), xmin=(0.0, 0.0, 0.0),
                   xmax=(1.0, 1.0, 1.0), metric=METRIC_MINKOWSKI, a=0.0, hslope=1.0,
                   gamma=gamma, cfl=cfl, t_final=t_final, recon=recon, floors=0,
                   bc=((BC_PERIODIC,) * 2,) * 3, P=P, info={"scale": scale})


# --------------------------------------------------------------------------
# Many uneven flat 2D grids (batched workload)
# --------------------------------------------------------------------------

BATCH_KINDS = ("slow", "alfven", "fast", "orszag_tang")
# integer wavenumber pairs (k = 2 pi (kx, ky) keeps the unit square periodic),
# oblique to the background field B = (1, 0, 0) so that the slow, Alfven and
# fast speeds are distinct and non-zero
BATCH_WAVENUMBERS = ((1, 1), (1, -1), (1, 2), (1, -2), (2, 1), (2, -1), (2, 2), (2, -2))


def batch_2d(ngrid: int = 64, nmin: int = 32, nmax: int = 256, seed: int = 0,
             t_final: float = 0.0) -> list:
    """``ngrid`` flat periodic square grids, N x N x 1 with N uniform in
    [nmin, nmax], in equal shares of slow, Alfven and fast linear modes and
    Orszag-Tang vortices (in a seeded order).  Modes: wavenumber pair drawn
    from BATCH_WAVENUMBERS, amplitude log-uniform in [1e-4, 1e-2]; Orszag-Tang:
    field scale s uniform in [0.5, 1.5].  Reconstruction MC or WENO5 with
    probability 1/2 each.  Every draw comes from splitmix_uniform(seed,
    8 g + field) for grid g, so grid g does not depend on ngrid."""
    idx = np.arange(8 * ngrid, dtype=np.uint64)
    u = splitmix_uniform(seed, idx).reshape(ngrid, 8)
    order = np.argsort(u[:, 0], kind="stable")
    kinds = [None] * ngrid
    for r, g in enumerate(order):
        kinds[g] = BATCH_KINDS[(r * len(BATCH_KINDS)) // ngrid]
    out = []
    for g in range(ngrid):
        n = min(nmin + int(u[g, 1] * (nmax - nmin + 1)), nmax)
        recon = RECON_WENO5 if u[g, 2] < 0.5 else RECON_MC
        if kinds[g] == "orszag_tang":
            pr = orszag_tang(n, scale=0.5 + u[g, 3], recon=recon, t_final=t_final)
        else:
            kx, ky = BATCH_WAVENUMBERS[min(int(u[g, 4] * len(BATCH_WAVENUMBERS)),
                                           len(BATCH_WAVENUMBERS) - 1)]
            amp = 10.0 ** (-4.0 + 2.0 * u[g, 5])
            pr = linear_mode(n, kinds[g], amp=amp, kvec=(2 * math.pi * kx, 2 * math.pi * ky),
                             recon=recon)
            pr.t_final = t_final
        pr.name = "g%02d_%s" % (g, pr.name)
        pr.info["kind"] = kinds[g]
        out.append(pr)
    return out


# --------------------------------------------------------------------------
# Arrival stream of the serving workload
# --------------------------------------------------------------------------

def serving_stream(nreq: int = 200, rate: float = 4.0, seed: int = 0) -> list:
    """``nreq`` requests arriving as a Poisson process of ``rate`` per second:
    60% Fishbone-Moncrief tori (spin a uniform in [0, 0.98], cubic N uniform
    in {64..192}), 40% Bondi inflows (cubic N, N uniform in {96..160}); each
    asks for a number of cycles uniform in {20..200} and runs in FP64 or in
    the mixed mode with probability 1/2.  Returns dicts (id, t_arrival,
    kind, n, a, steps, precision); ``serving_problem`` builds a request's
    input.  Draws: splitmix_uniform(seed, 8 r + field) for request r."""
    idx = np.arange(8 * nreq, dtype=np.uint64)
    u = splitmix_uniform(seed, idx).reshape(nreq, 8)
    t = 0.0
    out = []
    for r in range(nreq):
        t += -math.log(1.0 - u[r, 0]) / rate
        torus = u[r, 1] < 0.6
        if torus:
            n = 64 + min(int(u[r, 2] * 129), 128)
            a = 0.98 * u[r, 3]
        else:
            n = 96 + min(int(u[r, 2] * 65), 64)
            a = 0.0
        out.append({"id": r, "t_arrival": t, "kind": "torus" if torus else "bondi", "n": n, "a": a,
                    "steps": 20 + min(int(u[r, 4] * 181), 180), "precision": int(u[r, 5] < 0.5)})
    return out


def serving_problem(req: dict) -> "Problem":
    """The input of one serving request (see serving_stream)."""
    if req["kind"] == "torus":
        n = req["n"]
        pr = fm_torus(n, n, n, a=req["a"], seed=req["id"])
    else:
        pr = bondi(req["n"], req["n"], n3=req["n"])
    pr.precision = req["precision"]
    pr.name = "req%03d_%s" % (req["id"], pr.name)
    return pr


# --------------------------------------------------------------------------
# Kerr metric in modified Kerr-Schild coordinates (set-up only)
# --------------------------------------------------------------------------

def mks_theta(X2, h):
    return math.pi * X2 + 0.5 * (1.0 - h) * np.sin(2.0 * math.pi * X2)


def mks_gcov(r, X2, a, h):
    """g_{mu nu} of Kerr in MKS at (r, X2), arrays broadcast; shape (...,4,4)."""
    th = mks_theta(X2, h)
    s = np.sin(th)
    s = np.where(np.abs(s) < 1e-20, np.where(s >= 0, 1e-20, -1e-20), s)
    c = np.cos(th)
    s2, c2 = s * s, c * c
    sig = r * r + a * a * c2
    shape = np.broadcast(r, X2).shape
    g = np.zeros(shape + (4, 4))
    J = [np.ones(shape), r * np.ones(shape),
         math.pi * (1.0 + (1.0 - h) * np.cos(2.0 * math.pi * X2)) * np.ones(shape), np.ones(shape)]
    ks = np.zeros(shape + (4, 4))
    ks[..., 0, 0] = -(1.0 - 2.0 * r / sig)
    ks[..., 0, 1] = ks[..., 1, 0] = 2.0 * r / sig
    ks[..., 0, 3] = ks[..., 3, 0] = -2.0 * a * r * s2 / sig
    ks[..., 1, 1] = 1.0 + 2.0 * r / sig
    ks[..., 1, 3] = ks[..., 3, 1] = -a * s2 * (1.0 + 2.0 * r / sig)
    ks[..., 2, 2] = sig
    ks[..., 3, 3] = s2 * (sig + a * a * s2 * (1.0 + 2.0 * r / sig))
    for m in range(4):
        for nn in range(4):
            g[..., m, nn] = ks[..., m, nn] * J[m] * J[nn]
    return g


def mks_gdet(r, X2, a, h):
    """sqrt(-g) of Kerr in MKS, closed form: Sigma |sin theta| r dtheta/dX2."""
    th = mks_theta(X2, h)
    s = np.abs(np.sin(th))
    s = np.maximum(s, 1e-20)
    sig = r * r + a * a * np.cos(th) ** 2
    return sig * s * r * math.pi * (1.0 + (1.0 - h) * np.cos(2.0 * math.pi * X2))


def horizon_radius(a: float) -> float:
    return 1.0 + math.sqrt(1.0 - a * a)


def mks_rin(n1: int, a: float, r_out: float, zones_inside: float = 5.5) -> float:
    """Inner radius that puts `zones_inside` radial zones inside the horizon
    for log-uniform radial zones out to r_out."""
    rh = horizon_radius(a)
    return math.exp((n1 * math.log(rh) - zones_inside * math.log(r_out)) / (n1 - zones_inside))


# --------------------------------------------------------------------------
# Fishbone-Moncrief torus
# --------------------------------------------------------------------------

def fm_ell(a: float, r: float) -> float:
    """u^t u_phi of the prograde circular equatorial geodesic at r (Kerr,
    Boyer-Lindquist; Bardeen, Press & Teukolsky 1972)."""
    sr = math.sqrt(r)
    r32 = r * sr
    ut = (r32 + a) / (r ** 0.75 * math.sqrt(r32 - 3.0 * sr + 2.0 * a))
    uphi = (r * r - 2.0 * a * sr + a * a) / (r ** 0.75 * math.sqrt(r32 - 3.0 * sr + 2.0 * a))
    return ut * uphi


def fm_lnh(r, th, a, ell, r_in):
    """Fishbone-Moncrief log-enthalpy, zero at (r_in, pi/2)."""
    def raw(r, th):
        s = np.sin(th)
        c = np.cos(th)
        sig = r * r + a * a * c * c
        dlt = r * r - 2.0 * r + a * a
        A = (r * r + a * a) ** 2 - dlt * a * a * s * s
        q = np.sqrt(1.0 + 4.0 * ell * ell * sig * sig * dlt / (A * A * s * s))
        return 0.5 * np.log((1.0 + q) / (sig * dlt / A)) - 0.5 * q - 2.0 * a * r * ell / A
    return raw(r, th) - raw(np.asarray(r_in, dtype=float), np.asarray(math.pi / 2))


def fm_ucon_bl(r, th, a, ell):
    """(u^t, u^phi) of the FM torus in Boyer-Lindquist (u^r = u^th = 0),
    from the zero-angular-momentum-observer frame."""
    s = np.sin(th)
    c = np.cos(th)
    sig = r * r + a * a * c * c
    dlt = r * r - 2.0 * r + a * a
    A = (r * r + a * a) ** 2 - dlt * a * a * s * s
    em2chi = sig * sig * dlt / (A * A * s * s)
    up1 = np.sqrt((-1.0 + np.sqrt(1.0 + 4.0 * ell * ell * em2chi)) / 2.0)
    ut = np.sqrt(1.0 + up1 * up1) * np.sqrt(A / (sig * dlt))
    uphi = 2.0 * a * r * np.sqrt(1.0 + up1 * up1) / np.sqrt(A * sig * dlt) + \
        np.sqrt(sig / A) * up1 / s
    return ut, uphi


def _inv4(g):
    return np.linalg.inv(g)


def fm_torus(n1: int = 128, n2: int = 128, n3: int = 128, a: float = 0.9375, r_in: float = 6.0,
             r_max: float = 12.0, r_out: float = 50.0, hslope: float = 0.3, gamma: float = 4.0 / 3.0,
             kappa: float = 1e-3, beta: float = 100.0, pert: float = 0.04, seed: int = 0,
             recon: int = RECON_WENO5, cfl: float = 0.9, t_final: float = 0.0,
             field: bool = True) -> Problem:
    """3D Fishbone-Moncrief torus in MKS (X3 = phi over 2 pi)."""
    rin_grid = mks_rin(n1, a, r_out)
    x1min, x1max = math.log(rin_grid), math.log(r_out)
    dx1, dx2 = (x1max - x1min) / n1, 1.0 / n2
    ell = fm_ell(a, r_max)

    def torus_rho_u(r, X2):
        th = mks_theta(X2, hslope)
        with np.errstate(invalid="ignore", divide="ignore"):
            lnh = fm_lnh(r, th, a, ell, r_in)
        inside = (r >= r_in) & (lnh > 0.0) & np.isfinite(lnh)
        hh = np.exp(np.where(inside, lnh, 0.0))
        rho = np.where(inside, ((hh - 1.0) * (gamma - 1.0) / (kappa * gamma)) ** (1.0 / (gamma - 1.0)), 0.0)
        u = kappa * rho ** gamma / (gamma - 1.0)
        return rho, u, inside

    # zone centres (2D: the torus is axisymmetric)
    X1c = x1min + (np.arange(n1) + 0.5) * dx1
    X2c = (np.arange(n2) + 0.5) * dx2
    X1g, X2g = np.meshgrid(X1c, X2c, indexing="xy")   # [n2][n1]
    r = np.exp(X1g)
    th = mks_theta(X2g, hslope)
    rho, u, inside = torus_rho_u(r, X2g)
    rho_max = float(rho.max())
    rho = rho / rho_max
    u = u / rho_max

    # velocity: BL (u^t, 0, 0, u^phi) == KS components when u^r = 0; MKS u^3 = u^phi
    gcov = mks_gcov(r, X2g, a, hslope)
    gcon = _inv4(gcov)
    alpha = 1.0 / np.sqrt(-gcon[..., 0, 0])
    with np.errstate(invalid="ignore", divide="ignore"):
        ut_bl, uphi = fm_ucon_bl(r, th, a, ell)
    uphi = np.where(inside, uphi, 0.0)
    # normalise u^t in MKS for the (t, phi) velocity (same as BL since u^r = 0)
    g00, g03, g33 = gcov[..., 0, 0], gcov[..., 0, 3], gcov[..., 3, 3]
    # g00 ut^2 + 2 g03 ut uphi + g33 uphi^2 = -1  ->  positive root
    qa, qb, qc = g00, 2.0 * g03 * uphi, g33 * uphi * uphi + 1.0
    with np.errstate(invalid="ignore"):
        ut = (-qb - np.sqrt(qb * qb - 4.0 * qa * qc)) / (2.0 * qa)
    gam_n = alpha * ut
    util = np.zeros((3,) + r.shape)
    for i in range(3):
        ucon_i = uphi if i == 2 else 0.0
        util[i] = np.where(inside, ucon_i + gam_n * alpha * gcon[..., 0, i + 1], 0.0)

    # atmosphere at the floor values
    kk = 1.0 / (r * r * (1.0 + r / 10.0))
    rho_atm = 1e-6 * kk
    u_atm = 1e-8 * kk ** gamma
    rho2 = np.where(inside, rho, rho_atm)
    u2 = np.where(inside, u, u_atm)
    rho2 = np.maximum(rho2, rho_atm)
    u2 = np.maximum(u2, u_atm)

    P = np.zeros((NPRIM, n3, n2, n1))
    P[RHO] = rho2[None]
    P[UU] = u2[None]
    for i in range(3):
        P[U1 + i] = util[i][None]

    # seeded perturbation of u inside the torus (total spread of +-pert/2)
    if pert > 0.0:
        idx = np.arange(n1 * n2 * n3, dtype=np.uint64).reshape(n3, n2, n1)
        xi = splitmix_uniform(seed, idx)
        P[UU] = np.where(inside[None], P[UU] * (1.0 + pert * (xi - 0.5)), P[UU])

    if field:
        # A_phi at corners ~ max(rho/rho_max - 0.2, 0)
        X1k = x1min + np.arange(n1 + 1) * dx1
        X2k = np.arange(n2 + 1) * dx2
        X1kg, X2kg = np.meshgrid(X1k, X2k, indexing="xy")
        rk, _, _ = torus_rho_u(np.exp(X1kg), X2kg)
        Aphi = np.maximum(rk / rho_max - 0.2, 0.0)
        gd = mks_gdet(r, X2g, a, hslope)
        Bb1 = (Aphi[1:, :-1] + Aphi[1:, 1:] - Aphi[:-1, :-1] - Aphi[:-1, 1:]) / (2.0 * dx2 * gd)
        Bb2 = -(Aphi[:-1, 1:] + Aphi[1:, 1:] - Aphi[:-1, :-1] - Aphi[1:, :-1]) / (2.0 * dx1 * gd)
        # normalise: max P_gas / max P_b = beta (uses this module's own b^2)
        pg_max = float(((gamma - 1.0) * P[UU]).max())
        bsq = _bsq_mks(P[:, 0], Bb1, Bb2, gcov, gcon, alpha)
        pb_max = float((0.5 * bsq).max())
        norm = math.sqrt(pg_max / (beta * pb_max)) if pb_max > 0 else 0.0
        P[B1] = (norm * Bb1)[None]
        P[B2] = (norm * Bb2)[None]

    return Problem(
        name="fm_torus_%dx%dx%d" % (n1, n2, n3), n=(n1, n2, n3),
        xmin=(x1min, 0.0, 0.0), xmax=(x1max, 1.0, 2.0 * math.pi), metric=METRIC_MKS_KERR,
        a=a, hslope=hslope, gamma=gamma, cfl=cfl, t_final=t_final, recon=recon, floors=1,
        bc=((BC_OUTFLOW, BC_OUTFLOW), (BC_POLAR, BC_POLAR), (BC_PERIODIC, BC_PERIODIC)), P=P,
        info={"r_in_grid": rin_grid, "ell": ell, "rho_max_raw": rho_max, "r_in": r_in,
              "r_max": r_max, "r_out": r_out, "seed": seed, "beta": beta})


def _bsq_mks(P2, Bb1, Bb2, gcov, gcon, alpha):
    """b^2 of 2D primitive slices (set-up only)."""
    util = np.stack([P2[U1], P2[U2], P2[U3]], axis=-1)
    qsq = np.einsum("...i,...ij,...j->...", util, gcov[..., 1:, 1:], util)
    gam = np.sqrt(1.0 + qsq)
    ucon = np.zeros(P2[0].shape + (4,))
    ucon[..., 0] = gam / alpha
    for i in range(3):
        ucon[..., i + 1] = util[..., i] - gam * alpha * gcon[..., 0, i + 1]
    ucov = np.einsum("...ij,...j->...i", gcov, ucon)
    Bv = np.zeros(P2[0].shape + (4,))
    Bv[..., 1] = Bb1
    Bv[..., 2] = Bb2
    bt = np.einsum("...i,...i->...", Bv, ucov)
    bcon = (Bv + bt[..., None] * ucon) / ucon[..., 0:1]
    bcon[..., 0] = bt
    bcov = np.einsum("...ij,...j->...i", gcov, bcon)
    return np.einsum("...i,...i->...", bcon, bcov)


def random_states(n: int, seed: int = 0, metric: int = METRIC_MKS_KERR, a: float = 0.9375,
                  hslope: float = 0.3, gamma_max: float = 50.0, sigma_max: float = 400.0,
                  r_range=(1.2, 50.0)):
    """Random primitive states and coordinates for pointwise pins: rho in
    [1e-6, 1] (log-uniform), u in [1e-8, 10] (log-uniform), Lorentz factor up
    to gamma_max, b^2/rho up to sigma_max (by scaling B), random directions.
    Returns (X[n,4], P[n,8])."""
    rng = np.random.default_rng(seed)
    X = np.zeros((n, 4))
    if metric == METRIC_MKS_KERR:
        X[:, 1] = np.log(rng.uniform(r_range[0], r_range[1], n))
        X[:, 2] = rng.uniform(0.02, 0.98, n)
        X[:, 3] = rng.uniform(0, 2 * math.pi, n)
    else:
        X[:, 1:] = rng.uniform(0, 1, (n, 3))
    P = np.zeros((n, 8))
    P[:, RHO] = 10 ** rng.uniform(-6, 0, n)
    P[:, UU] = 10 ** rng.uniform(-8, 1, n)
    glf = 1.0 + (gamma_max - 1.0) * rng.uniform(0, 1, n) ** 3
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    mag = np.sqrt(glf * glf - 1.0)
    # utilde magnitude in an orthonormal-ish sense; exact gamma depends on the metric
    P[:, U1:U3 + 1] = d * mag[:, None]
    bd = rng.normal(size=(n, 3))
    P[:, B1:B3 + 1] = bd
    return X, P, rng.uniform(0, 1, n) * sigma_max


# --------------------------------------------------------------------------
# Michel (relativistic Bondi) inflow on Schwarzschild
# --------------------------------------------------------------------------

def michel_state(r, gamma=4.0 / 3.0, r_c=8.0, mdot=1.0):
    """Spherical polytropic inflow p = K rho^gamma onto a Schwarzschild black
    hole (M = 1) through the sonic radius r_c (Michel 1972).  With n =
    1/(gamma-1) and T = p/rho, the mass flux r^2 T^n u^r = -C1 and the
    Bernoulli constant (1 + (1+n) T)^2 (1 - 2/r + (u^r)^2) = C2 fix T(r) on
    the inflow branch; K follows from mdot = 4 pi r^2 rho |u^r|.
    Returns rho, u (internal energy density), u^r (< 0)."""
    r = np.asarray(r, dtype=float)
    n = 1.0 / (gamma - 1.0)
    uc2 = 1.0 / (2.0 * r_c)
    vc2 = uc2 / (1.0 - 3.0 * uc2)
    Tc = -n * vc2 / ((n + 1.0) * (n * vc2 - 1.0))
    C1 = math.sqrt(uc2) * r_c ** 2 * Tc ** n
    C2 = (1.0 + (1.0 + n) * Tc) ** 2 * (1.0 - 2.0 / r_c + uc2)

    lC2 = math.log(C2)

    def logF(T, rr):
        # log of the Bernoulli function; T -> 0 and T -> inf both send it up
        w = C1 / (rr * rr * T ** n)
        return 2.0 * math.log1p((1.0 + n) * T) + math.log(1.0 - 2.0 / rr + w * w)

    def dlogF(T, rr):  # derivative with respect to log T
        w = C1 / (rr * rr * T ** n)
        return (2.0 * (1.0 + n) * T / (1.0 + (1.0 + n) * T)
                - 2.0 * n * w * w / (1.0 - 2.0 / rr + w * w))

    def bisect(lo, hi, fun):
        flo = fun(lo)
        for _ in range(200):
            mid = math.sqrt(lo * hi)
            fm = fun(mid)
            if (fm > 0) == (flo > 0):
                lo, flo = mid, fm
            else:
                hi = mid
        return math.sqrt(lo * hi)

    T = np.empty_like(r)
    lo0, hi0 = Tc * 1e-12, Tc * 1e12
    for q, rr in np.ndenumerate(r):
        rr = float(rr)
        if rr <= 2.0:
            # inside the horizon 1 - 2/r + w^2 > 0 needs T below T_max, where the
            # function falls from +inf to -inf: one (supersonic) root
            tmax = (C1 / (rr * rr * math.sqrt(max(2.0 / rr - 1.0, 1e-300)))) ** (1.0 / n)
            T[q] = bisect(lo0, tmax * (1.0 - 1e-15), lambda t: logF(t, rr) - lC2)
            continue
        # the minimum over T of the Bernoulli function (sonic condition)
        tm = bisect(lo0, hi0, lambda t: dlogF(t, rr))
        if logF(tm, rr) >= lC2:
            T[q] = tm  # at the sonic radius (or within rounding of it)
            continue
        # the two roots of F = C2 straddle the minimum: the smaller T (faster
        # flow) is the supersonic branch taken inside r_c, the larger T outside
        if rr < r_c:
            T[q] = bisect(lo0, tm, lambda t: logF(t, rr) - lC2)
        else:
            T[q] = bisect(tm, hi0, lambda t: logF(t, rr) - lC2)
    ur = -C1 / (r * r * T ** n)
    Kn = 4.0 * math.pi * C1 / mdot  # rho = (T/K)^n with K^n = 4 pi C1 / mdot
    rho = T ** n / Kn
    u = n * rho * T
    return rho, u, ur


def bondi(n1: int = 64, n2: int = 64, r_out: float = 20.0, r_c: float = 8.0, mdot: float = 1.0,
          gamma: float = 4.0 / 3.0, hslope: float = 1.0, recon: int = RECON_MC, cfl: float = 0.9,
          t_final: float = 0.0, n3: int = 1, r_in: Optional[float] = None) -> Problem:
    """Stationary Michel inflow on Schwarzschild in MKS, n1 x n2 x n3 zones,
    inner radius r_in (default: 5.5 radial zones inside the horizon); the X1
    ghosts hold the analytic solution (BC_FIXED), X2 reflects at the poles,
    X3 periodic.  ``info['P_ghost']`` is the full array with ghosts for
    set_prims."""
    ng = 3
    a = 0.0
    rin = mks_rin(n1, a, r_out) if r_in is None else float(r_in)
    x1min, x1max = math.log(rin), math.log(r_out)
    dx1, dx2 = (x1max - x1min) / n1, 1.0 / n2
    X1 = x1min + (np.arange(-ng, n1 + ng) + 0.5) * dx1
    X2 = (np.arange(-ng, n2 + ng) + 0.5) * dx2
    X1g, X2g = np.meshgrid(X1, X2, indexing="xy")
    r = np.exp(X1g)
    rho1, u1d, ur1 = michel_state(np.exp(X1), gamma, r_c, mdot)
    rho = np.broadcast_to(rho1[None, :], r.shape)
    u = np.broadcast_to(u1d[None, :], r.shape)
    ur = np.broadcast_to(ur1[None, :], r.shape)
    g = mks_gcov(r, X2g, a, hslope)
    gcon = np.linalg.inv(g)
    alpha = 1.0 / np.sqrt(-gcon[..., 0, 0])
    u1 = ur / r  # MKS radial component
    # u^t from g_tt (u^t)^2 + 2 g_t1 u^t u^1 + g_11 (u^1)^2 = -1: the root that
    # stays finite through the horizon (g_tt = 0 there), in the form without
    # cancellation, 2 qc / (-qb + sqrt(qb^2 - 4 qa qc))  (-qb > 0 for inflow)
    qa, qb, qc = g[..., 0, 0], 2.0 * g[..., 0, 1] * u1, g[..., 1, 1] * u1 * u1 + 1.0
    ut = 2.0 * qc / (-qb + np.sqrt(qb * qb - 4.0 * qa * qc))
    gam_n = alpha * ut
    util1 = u1 + gam_n * alpha * gcon[..., 0, 1]
    util2 = gam_n * alpha * gcon[..., 0, 2]
    util3 = gam_n * alpha * gcon[..., 0, 3]
    s = (n3 + 2 * ng, n2 + 2 * ng, n1 + 2 * ng)
    Pg = np.zeros((NPRIM,) + s)
    for v, arr in ((RHO, rho), (UU, u), (U1, util1), (U2, util2), (U3, util3)):
        Pg[v] = arr[None]
    P = Pg[:, ng:-ng, ng:-ng, ng:-ng].copy()
    return Problem(
        name="bondi_%dx%dx%d" % (n1, n2, n3), n=(n1, n2, n3), xmin=(x1min, 0.0, 0.0),
        xmax=(x1max, 1.0, 2.0 * math.pi), metric=METRIC_MKS_KERR, a=a, hslope=hslope,
        gamma=gamma, cfl=cfl, t_final=t_final, recon=recon, floors=1,
        bc=((BC_FIXED, BC_FIXED), (BC_POLAR, BC_POLAR), (BC_PERIODIC, BC_PERIODIC)), P=P,
        info={"P_ghost": Pg, "r_c": r_c, "mdot": mdot, "r_in_grid": rin})
