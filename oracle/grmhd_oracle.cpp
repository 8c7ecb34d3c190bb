/*
 * grmhd_oracle.cpp -- plain, slow, scalar FP64 CPU oracle of the HARM
 * predictor-corrector GRMHD step (iharm3D, arXiv:2110.10191).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference for the
 * CUDA library.  Only tests/, __graft_entry__.smoke() and bench.py's oracle
 * leg (the CPU baseline, the reference arm and the accuracy figures measured
 * against the oracle) may load it.  It shares no code, header,
 * table or constant with the CUDA path (paper_2110_10191_gb300/csrc).
 *
 * What the paper fixes and what is read in:
 *   - Conservative finite-volume scheme on a logically Cartesian mesh in
 *     arbitrary stationary coordinates (paper, "Functionality and Purpose").
 *   - Flux-CT constrained transport, Toth (2000) (paper, "Implementation
 *     Notes", first paragraph).
 *   - Metric quantities evaluated numerically from the analytic line element
 *     (paper, "Implementation Notes", second paragraph): g_{mu nu} in closed
 *     form, g^{mu nu} by a 4x4 inverse, sqrt(-g) from the determinant and the
 *     connection by centred finite differences of g_{mu nu}.
 *   - 1D_W primitive recovery of Noble et al. (2006) (paper, "Implementation
 *     Notes", third paragraph).
 *   - Units GM = c = 1 (paper, "Implementation Notes", fourth paragraph).
 *   - The fluid bounds on rho, u, sigma, beta, u/rho and the Lorentz factor
 *     (paper, "Implementation Notes", bullet list of bounds).
 *   - Predictor-corrector stepping, MC / WENO5 reconstruction, local
 *     Lax-Friedrichs fluxes and fixup come from the HARM method the paper
 *     implements (Gammie, McKinney & Toth 2003); the paper does not print
 *     them.  Every point it leaves open is a stated reading (marked READING).
 *
 * Built twice: as liboracle.so (real == double) and, with -DORACLE_COUNT, as
 * liboracle_count.so where `real` counts every floating-point operation of
 * the step (add/sub, mul, div, sqrt; an FMA would count as 2) so that the
 * algorithmic FP64 work per zone-cycle is measured, not guessed.
 *
 * Compile with -ffp-contract=off so that no fused multiply-add is formed.
 */
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

/* ------------------------------------------------------------------------ */
/* The arithmetic type of the step.                                          */
/* ------------------------------------------------------------------------ */
#ifdef ORACLE_COUNT
struct OpCounts {
  double add, mul, div, sqrt;
};
/* phases: 0 face fluxes (from the reconstructed states), 1 boundary fixes +
 * flux-CT, 2 update + inversion + floors, 3 fixup, 4 anything else,
 * 5 reconstruction of the face states */
static OpCounts g_phase_ops[6];
static int g_phase = 4;
#define g_ops g_phase_ops[g_phase]
struct real {
  double v;
  real() : v(0.0) {}
  real(double x) : v(x) {}
};
static inline real operator+(real a, real b) { g_ops.add += 1; return real(a.v + b.v); }
static inline real operator-(real a, real b) { g_ops.add += 1; return real(a.v - b.v); }
static inline real operator*(real a, real b) { g_ops.mul += 1; return real(a.v * b.v); }
static inline real operator/(real a, real b) { g_ops.div += 1; return real(a.v / b.v); }
static inline real operator-(real a) { return real(-a.v); }
static inline real &operator+=(real &a, real b) { a = a + b; return a; }
static inline real &operator-=(real &a, real b) { a = a - b; return a; }
static inline real &operator*=(real &a, real b) { a = a * b; return a; }
static inline real &operator/=(real &a, real b) { a = a / b; return a; }
static inline bool operator<(real a, real b) { return a.v < b.v; }
static inline bool operator>(real a, real b) { return a.v > b.v; }
static inline bool operator<=(real a, real b) { return a.v <= b.v; }
static inline bool operator>=(real a, real b) { return a.v >= b.v; }
static inline bool operator==(real a, real b) { return a.v == b.v; }
static inline bool operator!=(real a, real b) { return a.v != b.v; }
static inline real rsqrt_(real a) { g_ops.sqrt += 1; return real(std::sqrt(a.v)); }
/* special functions (electron heating only) are counted with the square roots */
static inline real rpow(real a, real b) { g_ops.sqrt += 1; return real(std::pow(a.v, b.v)); }
static inline real rexp(real a) { g_ops.sqrt += 1; return real(std::exp(a.v)); }
static inline real rlog10(real a) { g_ops.sqrt += 1; return real(std::log10(a.v)); }
static inline real rabs(real a) { return real(std::fabs(a.v)); }
static inline double val(real a) { return a.v; }
static inline bool rfinite(real a) { return std::isfinite(a.v); }
#else
typedef double real;
static inline real rsqrt_(real a) { return std::sqrt(a); }
static inline real rpow(real a, real b) { return std::pow(a, b); }
static inline real rexp(real a) { return std::exp(a); }
static inline real rlog10(real a) { return std::log10(a); }
static inline real rabs(real a) { return std::fabs(a); }
static inline double val(real a) { return a; }
static inline bool rfinite(real a) { return std::isfinite(a); }
#endif

static inline real rmax(real a, real b) { return (a < b) ? b : a; }
static inline real rmin(real a, real b) { return (b < a) ? b : a; }

/* ------------------------------------------------------------------------ */
/* Layout and constants                                                      */
/* ------------------------------------------------------------------------ */
enum { RHO = 0, UU, U1, U2, U3, B1, B2, B3, NPRIM };
static const int NG = 3;                 /* ghost layers (WENO5 needs 3) */
enum { LOC_CENT = 0, LOC_FACE1, LOC_FACE2, NLOC }; /* FACE3 == CENT: X3-independent metrics */
enum { METRIC_MINKOWSKI = 0, METRIC_MKS_KERR = 1 };
enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_POLAR = 2, BC_FIXED = 3 };
enum { RECON_MC = 0, RECON_WENO5 = 1 };

/* Bounds (paper, "Implementation Notes", list of bounds). */
static const double FLOOR_RHO_K = 1.0e-6;    /* rho > 1e-6 k */
static const double FLOOR_U_K = 1.0e-8;      /* u > 1e-8 k^gamma */
static const double BSQ_OVER_RHO_MAX = 400.; /* sigma = b^2/rho < 400 */
static const double BETA_MIN = 2.5e-5;       /* beta = P_gas/P_b > 2.5e-5 */
static const double U_OVER_RHO_MAX = 100.;   /* u/rho < 100 */
static const double GAMMA_MAX = 50.;         /* Lorentz factor < 50 */
/* READING (drift-frame bounds): a field below this fraction of the density
 * has no direction worth following (see apply_floors_drift) */
static const double DRIFT_BSQ_MIN = 1.0e-20;

/* Electron thermodynamics (paper, "Implementation Notes": the optional
 * partition of dissipation between ions and electrons of Ressler et al.
 * (2015) with five heating models, and the bound P_gas/rho^gamma < 3 when
 * electron temperatures are evolved).  ELEC_CONSTANT (a fixed electron
 * share) is not one of the five; it serves the tests. */
enum {
  ELEC_OFF = 0, ELEC_CONSTANT = 1, ELEC_KAWAZURA = 2, ELEC_WERNER = 3, ELEC_ROWAN = 4,
  ELEC_SHARMA = 5, ELEC_HOWES = 6
};
static const double KTOT_MAX = 3.0;          /* P_gas / rho^gamma < 3 */
static const double ELEC_BETA_CAP = 1.0e20;  /* READING: beta of an unmagnetised zone */
static const double MP_OVER_ME = 1836.15267343; /* proton / electron mass */
struct ElecParams {
  int model;                  /* ELEC_* */
  double gam, game, gamp;     /* adiabatic index of the fluid, electrons, protons */
  double fel_const;           /* ELEC_CONSTANT's share */
  double tpte_min, tpte_max;  /* bounds on T_p / T_e */
};

/* floor flag bits */
enum {
  FF_GAMMA = 1, FF_RHO_GEOM = 2, FF_U_GEOM = 4, FF_SIGMA = 8, FF_BETA = 16, FF_TEMP = 32,
  FF_DRIFT = 64,       /* drift-frame bounds: the parcel was added and the sum inverted */
  FF_DRIFT_FAIL = 128, /* drift-frame bounds: that inversion failed, fluid-frame result kept */
  FF_KTOT = 256        /* electrons: u lowered to keep P_gas / rho^gamma below 3 */
};
enum { FLOOR_FLUID = 0, FLOOR_DRIFT = 1 };
/* inversion failure codes (first failing check, fixed order) */
enum {
  INV_OK = 0, INV_NOCONV = 1, INV_W_BAD = 2, INV_VSQ = 3, INV_RHO_NEG = 4, INV_U_NEG = 5, INV_D_NEG = 6
};

/* READING: 1D_W iteration rule.  Newton on W' = W - D (>= 0 for any physical
 * state) from the guess primitives, W' clamped to >= 0.  Stop after the
 * iteration whose step is <= 1e-8 W, followed by 1 extra Newton step (the
 * error after a step of 1e-8 W is of order 1e-16 W by quadratic convergence,
 * so one more step reaches round-off); at most 16 (+1) iterations.  A Newton step below W' = 0 halves W' instead.
 * An iterate with v^2(W) > 1 - 1e-10 (below the root, since v^2 falls with
 * W) is replaced by the bisection of the bracket [lo, hi] known from the
 * sign of f, or by doubling W while no upper end is known. */
static const int INV_MAXIT = 16;
static const int INV_EXTRA = 1;
static const double INV_TOL = 1.0e-8;
static const double INV_VSQ_MAX = 1.0 - 1.0e-10;

/* ------------------------------------------------------------------------ */
/* Geometry at one point                                                     */
/* ------------------------------------------------------------------------ */
struct GeomPt {
  real gcov[4][4], gcon[4][4];
  real gdet, alpha;
};

/* Closed-form metric g_{mu nu}(X).  Minkowski in Cartesian X, or Kerr in
 * Kerr-Schild form (mass 1, spin a) written in modified Kerr-Schild
 * coordinates r = exp(X1), theta = pi X2 + (1-h)/2 sin(2 pi X2), phi = X3
 * (paper: "coordinates adapted to place resolution", static mesh
 * refinement).  READING: |sin theta| is clamped to >= 1e-20 at the poles. */
static void metric_gcov(int kind, double a, double h, const double X[4], double g[4][4]) {
  for (int m = 0; m < 4; m++)
    for (int n = 0; n < 4; n++) g[m][n] = 0.0;
  if (kind == METRIC_MINKOWSKI) {
    g[0][0] = -1.0; g[1][1] = 1.0; g[2][2] = 1.0; g[3][3] = 1.0;
    return;
  }
  double r = std::exp(X[1]);
  double th = M_PI * X[2] + 0.5 * (1.0 - h) * std::sin(2.0 * M_PI * X[2]);
  double dr_dX1 = r;
  double dth_dX2 = M_PI * (1.0 + (1.0 - h) * std::cos(2.0 * M_PI * X[2]));
  double s = std::sin(th), c = std::cos(th);
  if (std::fabs(s) < 1e-20) s = (s >= 0.0) ? 1e-20 : -1e-20;
  double s2 = s * s, c2 = c * c;
  double sig = r * r + a * a * c2;
  double ks[4][4];
  for (int m = 0; m < 4; m++)
    for (int n = 0; n < 4; n++) ks[m][n] = 0.0;
  /* Kerr-Schild coordinates (t, r, theta, phi) */
  ks[0][0] = -(1.0 - 2.0 * r / sig);
  ks[0][1] = 2.0 * r / sig;
  ks[0][3] = -2.0 * a * r * s2 / sig;
  ks[1][1] = 1.0 + 2.0 * r / sig;
  ks[1][3] = -a * s2 * (1.0 + 2.0 * r / sig);
  ks[2][2] = sig;
  ks[3][3] = s2 * (sig + a * a * s2 * (1.0 + 2.0 * r / sig));
  ks[1][0] = ks[0][1]; ks[3][0] = ks[0][3]; ks[3][1] = ks[1][3];
  /* diagonal Jacobian dx^KS/dX^MKS */
  double J[4] = {1.0, dr_dX1, dth_dX2, 1.0};
  for (int m = 0; m < 4; m++)
    for (int n = 0; n < 4; n++) g[m][n] = ks[m][n] * J[m] * J[n];
}

/* 4x4 inverse by Gauss-Jordan elimination with partial pivoting; returns
 * the determinant. */
static double invert4(const double A[4][4], double inv[4][4]) {
  double M[4][8];
  for (int i = 0; i < 4; i++) {
    for (int j = 0; j < 4; j++) { M[i][j] = A[i][j]; M[i][4 + j] = (i == j) ? 1.0 : 0.0; }
  }
  double det = 1.0;
  for (int c = 0; c < 4; c++) {
    int piv = c;
    for (int r = c + 1; r < 4; r++)
      if (std::fabs(M[r][c]) > std::fabs(M[piv][c])) piv = r;
    if (piv != c) {
      for (int j = 0; j < 8; j++) { double t = M[c][j]; M[c][j] = M[piv][j]; M[piv][j] = t; }
      det = -det;
    }
    double p = M[c][c];
    det *= p;
    for (int j = 0; j < 8; j++) M[c][j] /= p;
    for (int r = 0; r < 4; r++) {
      if (r == c) continue;
      double f = M[r][c];
      for (int j = 0; j < 8; j++) M[r][j] -= f * M[c][j];
    }
  }
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) inv[i][j] = M[i][4 + j];
  return det;
}

/* gcon, sqrt(-g), lapse alpha = 1/sqrt(-g^{tt}) at X. */
static void geom_point(int kind, double a, double h, const double X[4], double gcov[4][4],
                       double gcon[4][4], double *gdet, double *alpha) {
  metric_gcov(kind, a, h, X, gcov);
  double det = invert4(gcov, gcon);
  *gdet = std::sqrt(std::fabs(det));
  *alpha = 1.0 / std::sqrt(-gcon[0][0]);
}

/* READING: finite-difference step of the numerical connection. */
static const double CONN_DELTA = 1.0e-5;

/* Connection Gamma^l_{m n} = 1/2 g^{l k} (d_m g_{k n} + d_n g_{k m} - d_k g_{m n})
 * with d_m by centred differences in X of step CONN_DELTA (d_t = 0: the
 * spacetime is stationary). */
static void conn_point(int kind, double a, double h, const double X[4], double conn[4][4][4]) {
  double gcov[4][4], gcon[4][4], gd, al;
  geom_point(kind, a, h, X, gcov, gcon, &gd, &al);
  double dg[4][4][4]; /* dg[m][k][n] = d_m g_{k n} */
  for (int k = 0; k < 4; k++)
    for (int n = 0; n < 4; n++) dg[0][k][n] = 0.0;
  for (int m = 1; m < 4; m++) {
    double Xp[4], Xm[4], gp[4][4], gm[4][4];
    for (int q = 0; q < 4; q++) { Xp[q] = X[q]; Xm[q] = X[q]; }
    Xp[m] += CONN_DELTA;
    Xm[m] -= CONN_DELTA;
    metric_gcov(kind, a, h, Xp, gp);
    metric_gcov(kind, a, h, Xm, gm);
    for (int k = 0; k < 4; k++)
      for (int n = 0; n < 4; n++) dg[m][k][n] = (gp[k][n] - gm[k][n]) / (2.0 * CONN_DELTA);
  }
  for (int l = 0; l < 4; l++)
    for (int m = 0; m < 4; m++)
      for (int n = 0; n < 4; n++) {
        double s = 0.0;
        for (int k = 0; k < 4; k++) s += gcon[l][k] * (dg[m][k][n] + dg[n][k][m] - dg[k][m][n]);
        conn[l][m][n] = 0.5 * s;
      }
}

/* ------------------------------------------------------------------------ */
/* Fluid state at a point: u^mu, u_mu, b^mu, b_mu (HARM's primitives).        */
/* ------------------------------------------------------------------------ */
struct FluidState {
  real ucon[4], ucov[4], bcon[4], bcov[4], bsq;
};

static inline void lower(const real con[4], const GeomPt &g, real cov[4]) {
  for (int m = 0; m < 4; m++) {
    real s = 0.0;
    for (int n = 0; n < 4; n++) s += g.gcov[m][n] * con[n];
    cov[m] = s;
  }
}

/* u^t = gamma/alpha, u^i = utilde^i - gamma alpha g^{ti},
 * gamma = sqrt(1 + g_ij utilde^i utilde^j). */
static void ucon_calc(const real P[NPRIM], const GeomPt &g, real ucon[4]) {
  real qsq = 0.0;
  for (int i = 1; i < 4; i++)
    for (int j = 1; j < 4; j++) qsq += g.gcov[i][j] * P[U1 + i - 1] * P[U1 + j - 1];
  real gamma = rsqrt_(1.0 + qsq);
  ucon[0] = gamma / g.alpha;
  for (int i = 1; i < 4; i++) ucon[i] = P[U1 + i - 1] - gamma * g.alpha * g.gcon[0][i];
}

/* u_mu from utilde directly (the normal observer has n_i = 0):
 * u_i = g_ij utilde^j and u_t = -alpha gamma + g_tj utilde^j.  Equal to
 * g_{mu nu} u^nu, without the cancellation between the shift terms that the
 * contraction suffers for slow flows in Kerr-Schild coordinates. */
static void ucov_calc(const real P[NPRIM], const GeomPt &g, const real ucon[4], real ucov[4]) {
  real gamma = ucon[0] * g.alpha;
  for (int i = 1; i < 4; i++) {
    real s = 0.0;
    for (int j = 1; j < 4; j++) s += g.gcov[i][j] * P[U1 + j - 1];
    ucov[i] = s;
  }
  real s0 = -g.alpha * gamma;
  for (int j = 1; j < 4; j++) s0 += g.gcov[0][j] * P[U1 + j - 1];
  ucov[0] = s0;
}

/* b^t = B^i u_i, b^i = (B^i + b^t u^i)/u^t, with B^i = *F^{it}. */
static void get_state(const real P[NPRIM], const GeomPt &g, FluidState &s) {
  ucon_calc(P, g, s.ucon);
  ucov_calc(P, g, s.ucon, s.ucov);
  s.bcon[0] = 0.0;
  for (int i = 1; i < 4; i++) s.bcon[0] += P[B1 + i - 1] * s.ucov[i];
  for (int i = 1; i < 4; i++) s.bcon[i] = (P[B1 + i - 1] + s.bcon[0] * s.ucon[i]) / s.ucon[0];
  lower(s.bcon, g, s.bcov);
  s.bsq = 0.0;
  for (int m = 0; m < 4; m++) s.bsq += s.bcon[m] * s.bcov[m];
}

/* T^mu_nu = (rho + u + p + b^2) u^mu u_nu + (p + b^2/2) delta^mu_nu - b^mu b_nu */
static void mhd_row(const real P[NPRIM], const FluidState &s, real gam, int mu, real T[4]) {
  real pgas = (gam - 1.0) * P[UU];
  real w = P[RHO] + P[UU] + pgas + s.bsq;
  real ptot = pgas + 0.5 * s.bsq;
  for (int nu = 0; nu < 4; nu++) {
    T[nu] = w * s.ucon[mu] * s.ucov[nu] - s.bcon[mu] * s.bcov[nu];
    if (nu == mu) T[nu] += ptot;
  }
}

/* Conserved densities (dir 0) or fluxes (dir 1..3), all sqrt(-g)-weighted:
 *   rho u^d ;  T^d_t + rho u^d (rest mass subtracted: HARM convention) ;
 *   T^d_i ;  b^j u^d - b^d u^j. */
static void prim_to_flux(const real P[NPRIM], const FluidState &s, const GeomPt &g, real gam,
                         int dir, real F[NPRIM]) {
  real T[4];
  mhd_row(P, s, gam, dir, T);
  F[RHO] = P[RHO] * s.ucon[dir];
  F[UU] = T[0] + F[RHO];
  F[U1] = T[1];
  F[U2] = T[2];
  F[U3] = T[3];
  for (int j = 1; j < 4; j++) F[B1 + j - 1] = s.bcon[j] * s.ucon[dir] - s.bcon[dir] * s.ucon[j];
  for (int v = 0; v < NPRIM; v++) F[v] *= g.gdet;
}

/* Fast-magnetosonic coordinate speeds along dir.  A wave covector
 * k = A - v B with A_mu = delta^dir_mu, B_mu = delta^t_mu satisfies
 * (k.u)^2 = c_ms^2 [k.k + (k.u)^2], with
 * c_ms^2 = c_s^2 + v_A^2 - c_s^2 v_A^2 (HARM's upper bound on the fast speed).
 * READING: a negative discriminant is set to zero. */
static void vchar(const real P[NPRIM], const FluidState &s, const GeomPt &g, real gam, int dir,
                  real *vmax, real *vmin) {
  real ef = P[RHO] + gam * P[UU];
  real ee = s.bsq + ef;
  real va2 = s.bsq / ee;
  real cs2 = gam * (gam - 1.0) * P[UU] / ef;
  real cms2 = cs2 + va2 - cs2 * va2;
  real Asq = g.gcon[dir][dir];
  real Bsq = g.gcon[0][0];
  real AB = g.gcon[0][dir];
  real Au = s.ucon[dir];
  real Bu = s.ucon[0];
  real qa = Bu * Bu - (Bsq + Bu * Bu) * cms2;
  real qb = -2.0 * (Au * Bu - (AB + Au * Bu) * cms2);
  real qc = Au * Au - (Asq + Au * Au) * cms2;
  real disc = qb * qb - 4.0 * qa * qc;
  if (disc < 0.0) disc = 0.0;
  disc = rsqrt_(disc);
  real v1 = (-qb + disc) / (2.0 * qa);
  real v2 = (-qb - disc) / (2.0 * qa);
  *vmax = rmax(v1, v2);
  *vmin = rmin(v1, v2);
}

/* ------------------------------------------------------------------------ */
/* Reconstruction                                                            */
/* ------------------------------------------------------------------------ */
/* Monotonized-central limited slope: minmod(2 dm, (dm+dp)/2, 2 dp), zero
 * where the one-sided differences change sign.  Face values y -/+ slope/2. */
static real mc_slope(real x0, real x1, real x2) {
  real dm = x1 - x0, dp = x2 - x1;
  real slope = 0.0;
  if (dm * dp > 0.0) {
    real dc = 0.5 * (dm + dp);
    real m = rmin(rmin(rabs(2.0 * dm), rabs(dc)), rabs(2.0 * dp));
    slope = (dc > 0.0) ? m : -m;
  }
  return slope;
}

static void recon_mc(real x0, real x1, real x2, real *lout, real *rout) {
  real slope = mc_slope(x0, x1, x2);
  *lout = x1 - 0.5 * slope;
  *rout = x1 + 0.5 * slope;
}

/* Jiang-Shu WENO5 value at the right face of the middle zone of
 * x0..x4 (zones i-2..i+2).  READING: epsilon = 1e-26, weights ~ 1/(eps+beta)^2. */
static real weno5_right(real x0, real x1, real x2, real x3, real x4) {
  const real eps = 1.0e-26;
  real q0 = (2.0 * x0 - 7.0 * x1 + 11.0 * x2) / 6.0;
  real q1 = (-x1 + 5.0 * x2 + 2.0 * x3) / 6.0;
  real q2 = (2.0 * x2 + 5.0 * x3 - x4) / 6.0;
  real t;
  real b0 = (13.0 / 12.0) * (x0 - 2.0 * x1 + x2) * (x0 - 2.0 * x1 + x2);
  t = x0 - 4.0 * x1 + 3.0 * x2;
  b0 += 0.25 * t * t;
  real b1 = (13.0 / 12.0) * (x1 - 2.0 * x2 + x3) * (x1 - 2.0 * x2 + x3);
  t = x1 - x3;
  b1 += 0.25 * t * t;
  real b2 = (13.0 / 12.0) * (x2 - 2.0 * x3 + x4) * (x2 - 2.0 * x3 + x4);
  t = 3.0 * x2 - 4.0 * x3 + x4;
  b2 += 0.25 * t * t;
  real a0 = 0.1 / ((eps + b0) * (eps + b0));
  real a1 = 0.6 / ((eps + b1) * (eps + b1));
  real a2 = 0.3 / ((eps + b2) * (eps + b2));
  real sum = a0 + a1 + a2;
  return (a0 * q0 + a1 * q1 + a2 * q2) / sum;
}

static void recon_weno5(const real x[5], real *lout, real *rout) {
  *rout = weno5_right(x[0], x[1], x[2], x[3], x[4]);
  *lout = weno5_right(x[4], x[3], x[2], x[1], x[0]);
}

/* Both WENO5 face values of the middle zone of x0..x4 from one set of
 * smoothness indicators (the reconstruction step produces a zone's two
 * interface values from the zone's own stencil).  The high face weighs the
 * candidates (2x0 - 7x1 + 11x2)/6, (-x1 + 5x2 + 2x3)/6, (2x2 + 5x3 - x4)/6
 * by 0.1, 0.6, 0.3 over (eps + beta_k)^2 with beta_0, beta_1, beta_2; the
 * low face is its mirror image: candidates (2x4 - 7x3 + 11x2)/6,
 * (-x3 + 5x2 + 2x1)/6, (2x2 + 5x1 - x0)/6 with beta_2, beta_1, beta_0 (a
 * three-zone indicator reads the same in either direction).  The values
 * are weno5_right's, each indicator formed once; every term is written in
 * a mirror-symmetric order, so reversing the stencil swaps the two face
 * values exactly. */
static void weno5_zone(const real x[5], real *lout, real *rout) {
  const real eps = 1.0e-26;
  real t, s;
  t = (x[0] + x[2]) - 2.0 * x[1];
  s = (3.0 * x[2] - 4.0 * x[1]) + x[0];
  real e0 = eps + ((13.0 / 12.0) * t * t + 0.25 * s * s);
  t = (x[1] + x[3]) - 2.0 * x[2];
  s = x[1] - x[3];
  real e1 = eps + ((13.0 / 12.0) * t * t + 0.25 * s * s);
  t = (x[2] + x[4]) - 2.0 * x[3];
  s = (3.0 * x[2] - 4.0 * x[3]) + x[4];
  real e2 = eps + ((13.0 / 12.0) * t * t + 0.25 * s * s);
  e0 = e0 * e0;
  e1 = e1 * e1;
  e2 = e2 * e2;
  /* high face */
  real a0 = 0.1 / e0, a1 = 0.6 / e1, a2 = 0.3 / e2;
  real q0 = (2.0 * x[0] - 7.0 * x[1] + 11.0 * x[2]) / 6.0;
  real q1 = (-x[1] + 5.0 * x[2] + 2.0 * x[3]) / 6.0;
  real q2 = (2.0 * x[2] + 5.0 * x[3] - x[4]) / 6.0;
  *rout = (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
  /* low face */
  a0 = 0.1 / e2;
  a1 = 0.6 / e1;
  a2 = 0.3 / e0;
  q0 = (2.0 * x[4] - 7.0 * x[3] + 11.0 * x[2]) / 6.0;
  q1 = (-x[3] + 5.0 * x[2] + 2.0 * x[1]) / 6.0;
  q2 = (2.0 * x[2] + 5.0 * x[1] - x[0]) / 6.0;
  *lout = (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

/* ------------------------------------------------------------------------ */
/* Simulation state                                                          */
/* ------------------------------------------------------------------------ */
struct Sim {
  int n[3];
  int s[3];
  long ntot;
  double xmin[3], xmax[3], dx[3];
  int metric;
  double a, hslope;
  double gam, cfl, t_final;
  int recon, floors_on;
  int floor_frame; /* FLOOR_FLUID or FLOOR_DRIFT */
  int elec;          /* electron model (ELEC_*), 0: off */
  ElecParams ep;
  int bc[3][2];
  std::vector<GeomPt> geom[NLOC];       /* [ij] */
  std::vector<real> conn;               /* [ij][4][4][4] */
  std::vector<real> rho_floor, u_floor; /* [ij] floor thresholds */
  std::vector<real> P, Ph;              /* [v][k][j][i] */
  std::vector<real> F[3];               /* [v][k][j][i], face i-1/2 etc. */
  /* electrons: K = (kappa_tot, kappa_e) = (P_gas / rho^gamma, P_e / rho^gamma_e)
   * per zone, [s][k][j][i], and their fluxes; stage arrays as P, Ph */
  std::vector<real> K, Kh, FK[3];
  std::vector<real> Lz, Rz, KLz, KRz; /* scratch: zones' face values along one direction */
  std::vector<real> emf[3];
  std::vector<int> pflag, fflag;
  real ctop_max[3];
  double t, dt, dt_prev;
  long nstep;
  long inv_fail_total, floor_hits_total, unrecoverable_total;
};

static inline long IDX(const Sim *S, int i, int j, int k) {
  return ((long)k * S->s[1] + j) * S->s[0] + i;
}
static inline long IJ(const Sim *S, int i, int j) { return (long)j * S->s[0] + i; }

static double xcent(const Sim *S, int d, int i) { return S->xmin[d] + (i - NG + 0.5) * S->dx[d]; }
static double xface(const Sim *S, int d, int i) { return S->xmin[d] + (i - NG) * S->dx[d]; }

static void build_geometry(Sim *S) {
  long n2d = (long)S->s[0] * S->s[1];
  for (int l = 0; l < NLOC; l++) S->geom[l].assign(n2d, GeomPt());
  S->conn.assign(n2d * 64, real(0.0));
  S->rho_floor.assign(n2d, real(0.0));
  S->u_floor.assign(n2d, real(0.0));
  for (int j = 0; j < S->s[1]; j++)
    for (int i = 0; i < S->s[0]; i++) {
      for (int l = 0; l < NLOC; l++) {
        double X[4] = {0.0, xcent(S, 0, i), xcent(S, 1, j), 0.0};
        if (l == LOC_FACE1) X[1] = xface(S, 0, i);
        if (l == LOC_FACE2) X[2] = xface(S, 1, j);
        double gcov[4][4], gcon[4][4], gd, al;
        geom_point(S->metric, S->a, S->hslope, X, gcov, gcon, &gd, &al);
        GeomPt &G = S->geom[l][IJ(S, i, j)];
        for (int m = 0; m < 4; m++)
          for (int n = 0; n < 4; n++) { G.gcov[m][n] = gcov[m][n]; G.gcon[m][n] = gcon[m][n]; }
        G.gdet = gd;
        G.alpha = al;
        if (l == LOC_CENT) {
          double cn[4][4][4];
          conn_point(S->metric, S->a, S->hslope, X, cn);
          real *c = &S->conn[IJ(S, i, j) * 64];
          for (int q = 0; q < 64; q++) c[q] = (&cn[0][0][0])[q];
          if (S->metric == METRIC_MKS_KERR) {
            /* k = 1/(r^2 (1 + r/10)) with r the radial coordinate */
            double r = std::exp(X[1]);
            double kk = 1.0 / (r * r * (1.0 + r / 10.0));
            S->rho_floor[IJ(S, i, j)] = FLOOR_RHO_K * kk;
            S->u_floor[IJ(S, i, j)] = FLOOR_U_K * std::pow(kk, S->gam);
          }
        }
      }
    }
}

/* ------------------------------------------------------------------------ */
/* Boundary conditions (ghost fill).  READING: X1 outflow copies the last      */
/* active zone, rescales B^i by sqrt(-g) so sqrt(-g) B^i is constant, and     */
/* zeroes utilde^1 where it points into the domain (the inflow check).  X2    */
/* polar reflection copies the mirror zone with utilde^2 and B^2 negated.     */
/* Order X1 (interior j,k), X2 (all i), X3 (all i,j) fills edges/corners.     */
/* ------------------------------------------------------------------------ */
/* periodic image of ghost index g along a direction of n zones */
static int wrap_index(int g, int n) {
  int q = (g - NG) % n;
  if (q < 0) q += n;
  return NG + q;
}

/* K (may be empty): the electron entropies, copied as scalars */
static void copy_zone(Sim *S, std::vector<real> &P, std::vector<real> &K, long dst, long src) {
  for (int v = 0; v < NPRIM; v++) P[v * S->ntot + dst] = P[v * S->ntot + src];
  if (!K.empty())
    for (int q = 0; q < 2; q++) K[q * S->ntot + dst] = K[q * S->ntot + src];
}

static void bounds(Sim *S, std::vector<real> &P, std::vector<real> &K) {
  const long N = S->ntot;
  const int n1 = S->n[0], n2 = S->n[1], n3 = S->n[2];
  /* X1 */
  for (int k = NG; k < n3 + NG; k++)
    for (int j = NG; j < n2 + NG; j++)
      for (int g = 0; g < NG; g++) {
        /* lower */
        int ig = g, ia;
        if (S->bc[0][0] == BC_PERIODIC) {
          copy_zone(S, P, K, IDX(S, ig, j, k), IDX(S, wrap_index(ig, n1), j, k));
        } else if (S->bc[0][0] == BC_OUTFLOW) {
          ia = NG;
          long d = IDX(S, ig, j, k), s = IDX(S, ia, j, k);
          copy_zone(S, P, K, d, s);
          real rescale = S->geom[LOC_CENT][IJ(S, ia, j)].gdet / S->geom[LOC_CENT][IJ(S, ig, j)].gdet;
          for (int b = B1; b <= B3; b++) P[b * N + d] *= rescale;
          if (P[U1 * N + d] > 0.0) P[U1 * N + d] = 0.0;
        }
        /* upper */
        ig = n1 + NG + g;
        if (S->bc[0][1] == BC_PERIODIC) {
          copy_zone(S, P, K, IDX(S, ig, j, k), IDX(S, wrap_index(ig, n1), j, k));
        } else if (S->bc[0][1] == BC_OUTFLOW) {
          ia = n1 + NG - 1;
          long d = IDX(S, ig, j, k), s = IDX(S, ia, j, k);
          copy_zone(S, P, K, d, s);
          real rescale = S->geom[LOC_CENT][IJ(S, ia, j)].gdet / S->geom[LOC_CENT][IJ(S, ig, j)].gdet;
          for (int b = B1; b <= B3; b++) P[b * N + d] *= rescale;
          if (P[U1 * N + d] < 0.0) P[U1 * N + d] = 0.0;
        }
      }
  /* X2 */
  for (int k = NG; k < n3 + NG; k++)
    for (int i = 0; i < S->s[0]; i++)
      for (int g = 0; g < NG; g++) {
        int jg = NG - 1 - g;
        if (S->bc[1][0] == BC_PERIODIC) {
          copy_zone(S, P, K, IDX(S, i, jg, k), IDX(S, i, wrap_index(jg, n2), k));
        } else if (S->bc[1][0] == BC_POLAR) {
          long d = IDX(S, i, jg, k);
          copy_zone(S, P, K, d, IDX(S, i, NG + g, k));
          P[U2 * N + d] = -P[U2 * N + d];
          P[B2 * N + d] = -P[B2 * N + d];
        } else if (S->bc[1][0] == BC_OUTFLOW) {
          copy_zone(S, P, K, IDX(S, i, jg, k), IDX(S, i, NG, k));
        }
        jg = n2 + NG + g;
        if (S->bc[1][1] == BC_PERIODIC) {
          copy_zone(S, P, K, IDX(S, i, jg, k), IDX(S, i, wrap_index(jg, n2), k));
        } else if (S->bc[1][1] == BC_POLAR) {
          long d = IDX(S, i, jg, k);
          copy_zone(S, P, K, d, IDX(S, i, n2 + NG - 1 - g, k));
          P[U2 * N + d] = -P[U2 * N + d];
          P[B2 * N + d] = -P[B2 * N + d];
        } else if (S->bc[1][1] == BC_OUTFLOW) {
          copy_zone(S, P, K, IDX(S, i, jg, k), IDX(S, i, n2 + NG - 1, k));
        }
      }
  /* X3 */
  for (int j = 0; j < S->s[1]; j++)
    for (int i = 0; i < S->s[0]; i++)
      for (int g = 0; g < NG; g++) {
        int kg = NG - 1 - g;
        if (S->bc[2][0] == BC_PERIODIC)
          copy_zone(S, P, K, IDX(S, i, j, kg), IDX(S, i, j, wrap_index(kg, n3)));
        else if (S->bc[2][0] == BC_OUTFLOW)
          copy_zone(S, P, K, IDX(S, i, j, kg), IDX(S, i, j, NG));
        kg = n3 + NG + g;
        if (S->bc[2][1] == BC_PERIODIC)
          copy_zone(S, P, K, IDX(S, i, j, kg), IDX(S, i, j, wrap_index(kg, n3)));
        else if (S->bc[2][1] == BC_OUTFLOW)
          copy_zone(S, P, K, IDX(S, i, j, kg), IDX(S, i, j, n3 + NG - 1));
      }
}

/* ------------------------------------------------------------------------ */
/* Face fluxes: reconstruction + LLF, over the face range flux-CT needs       */
/* (one extra transverse layer on each side).                                 */
/* ------------------------------------------------------------------------ */
static void load_prims(const Sim *S, const std::vector<real> &P, long id, real out[NPRIM]) {
  for (int v = 0; v < NPRIM; v++) out[v] = P[v * S->ntot + id];
}

/* The two face values along d of every zone that the faces lo..hi need
 * (zones lo[d]-1 .. hi[d] along d, the faces' transverse ranges), for the
 * nvar variables of A: Lz at the zone's low face, Rz at its high face, each
 * zone reconstructed once from its own stencil (MC slope or WENO5 pair). */
static void zone_faces(const Sim *S, const std::vector<real> &A, int nvar, int d, const int lo[3],
                       const int hi[3], std::vector<real> &Lz, std::vector<real> &Rz) {
  const long N = S->ntot;
  int off[3] = {0, 0, 0};
  off[d] = 1;
  int zlo[3] = {lo[0], lo[1], lo[2]};
  zlo[d] = lo[d] - 1;
  for (int k = zlo[2]; k <= hi[2]; k++)
    for (int j = zlo[1]; j <= hi[1]; j++)
      for (int i = zlo[0]; i <= hi[0]; i++) {
        long c = IDX(S, i, j, k);
        for (int v = 0; v < nvar; v++) {
          real x[5]; /* zones c-2 .. c+2 along d */
          for (int q = 0; q < 5; q++) {
            int sft = q - 2;
            x[q] = A[v * N + IDX(S, i + sft * off[0], j + sft * off[1], k + sft * off[2])];
          }
          real l, r;
          if (S->recon == RECON_WENO5)
            weno5_zone(x, &l, &r);
          else
            recon_mc(x[1], x[2], x[3], &l, &r);
          Lz[v * N + c] = l;
          Rz[v * N + c] = r;
        }
      }
}

/* Local Lax-Friedrichs flux at one face; returns ctop. */
static real llf_face(const Sim *S, const GeomPt &g, int d, const real PL[NPRIM],
                     const real PR[NPRIM], real Fout[NPRIM]) {
  FluidState sL, sR;
  get_state(PL, g, sL);
  get_state(PR, g, sR);
  real FL[NPRIM], FR[NPRIM], UL[NPRIM], UR[NPRIM];
  prim_to_flux(PL, sL, g, S->gam, d + 1, FL);
  prim_to_flux(PR, sR, g, S->gam, d + 1, FR);
  prim_to_flux(PL, sL, g, S->gam, 0, UL);
  prim_to_flux(PR, sR, g, S->gam, 0, UR);
  real vmaxL, vminL, vmaxR, vminR;
  vchar(PL, sL, g, S->gam, d + 1, &vmaxL, &vminL);
  vchar(PR, sR, g, S->gam, d + 1, &vmaxR, &vminR);
  real cmax = rmax(rmax(real(0.0), vmaxL), vmaxR);
  real cmin = rmax(rmax(real(0.0), -vminL), -vminR);
  real ctop = rmax(cmax, cmin);
  for (int v = 0; v < NPRIM; v++)
    Fout[v] = 0.5 * (FL[v] + FR[v] - ctop * (UR[v] - UL[v]));
  return ctop;
}

/* Fluxes of the electron entropies (Ressler et al. 2015): kappa_tot and
 * kappa_e are carried with the mass, conserved density sqrt(-g) rho u^t K
 * and flux sqrt(-g) rho u^d K, combined as the other fluxes are (local
 * Lax-Friedrichs with the face's ctop) from K reconstructed on each side
 * (KL[q], KR[q]). */
static void elec_face(const GeomPt &g, int d, const real PL[NPRIM], const real PR[NPRIM],
                      real ctop, const real KL[2], const real KR[2], real FK[2]) {
  FluidState sL, sR;
  get_state(PL, g, sL);
  get_state(PR, g, sR);
  real mL = PL[RHO] * sL.ucon[d + 1], mR = PR[RHO] * sR.ucon[d + 1]; /* rho u^d */
  real dL = PL[RHO] * sL.ucon[0], dR = PR[RHO] * sR.ucon[0];         /* rho u^t */
  for (int q = 0; q < 2; q++)
    FK[q] = 0.5 * g.gdet * (mL * KL[q] + mR * KR[q] - ctop * (dR * KR[q] - dL * KL[q]));
}

static void get_fluxes(Sim *S, const std::vector<real> &P, const std::vector<real> &K) {
  const long N = S->ntot;
  for (int d = 0; d < 3; d++) {
    S->ctop_max[d] = 0.0;
    int lo[3], hi[3]; /* inclusive ranges */
    for (int e = 0; e < 3; e++) { lo[e] = NG - 1; hi[e] = S->n[e] + NG; }
    lo[d] = NG;
    hi[d] = S->n[d] + NG;
    int loc = (d == 0) ? LOC_FACE1 : (d == 1) ? LOC_FACE2 : LOC_CENT;
    /* every zone's two face values along d, then the faces */
#ifdef ORACLE_COUNT
    int saved = g_phase;
    g_phase = 5;
#endif
    zone_faces(S, P, NPRIM, d, lo, hi, S->Lz, S->Rz);
    if (S->elec) zone_faces(S, K, 2, d, lo, hi, S->KLz, S->KRz);
#ifdef ORACLE_COUNT
    g_phase = saved;
#endif
    const long st = (d == 0) ? 1 : (d == 1) ? S->s[0] : (long)S->s[0] * S->s[1];
    for (int k = lo[2]; k <= hi[2]; k++)
      for (int j = lo[1]; j <= hi[1]; j++)
        for (int i = lo[0]; i <= hi[0]; i++) {
          real PL[NPRIM], PR[NPRIM], Fo[NPRIM];
          const long c = IDX(S, i, j, k);
          for (int v = 0; v < NPRIM; v++) {
            PL[v] = S->Rz[v * N + c - st]; /* high face of the zone below the face */
            PR[v] = S->Lz[v * N + c];      /* low face of the zone above it */
          }
          const GeomPt &g = S->geom[loc][IJ(S, i, j)];
          real ctop = llf_face(S, g, d, PL, PR, Fo);
          long id = IDX(S, i, j, k);
          for (int v = 0; v < NPRIM; v++) S->F[d][v * N + id] = Fo[v];
          if (S->elec) {
            real KL[2], KR[2], FK[2];
            for (int q = 0; q < 2; q++) {
              KL[q] = S->KRz[q * N + c - st];
              KR[q] = S->KLz[q * N + c];
            }
            elec_face(g, d, PL, PR, ctop, KL, KR, FK);
            for (int q = 0; q < 2; q++) S->FK[d][q * N + id] = FK[q];
          }
          /* dt uses the faces of interior zones only */
          bool interior = true;
          for (int e = 0; e < 3; e++) {
            if (e == d) continue;
            int c = (e == 0) ? i : (e == 1) ? j : k;
            if (c < NG || c >= S->n[e] + NG) interior = false;
          }
          if (interior && ctop > S->ctop_max[d]) S->ctop_max[d] = ctop;
        }
  }
}

/* READING (boundary flux fixes): X2 polar faces carry no flux; at an X1
 * outflow boundary no mass flows in from outside, nor do the electron
 * entropies that the mass carries. */
static void fix_flux(Sim *S) {
  const long N = S->ntot;
  if (S->bc[1][0] == BC_POLAR || S->bc[1][1] == BC_POLAR) {
    for (int k = NG - 1; k <= S->n[2] + NG; k++)
      for (int i = NG - 1; i <= S->n[0] + NG; i++) {
        if (S->bc[1][0] == BC_POLAR) {
          for (int v = 0; v < NPRIM; v++) S->F[1][v * N + IDX(S, i, NG, k)] = 0.0;
          if (S->elec)
            for (int q = 0; q < 2; q++) S->FK[1][q * N + IDX(S, i, NG, k)] = 0.0;
        }
        if (S->bc[1][1] == BC_POLAR) {
          for (int v = 0; v < NPRIM; v++) S->F[1][v * N + IDX(S, i, S->n[1] + NG, k)] = 0.0;
          if (S->elec)
            for (int q = 0; q < 2; q++) S->FK[1][q * N + IDX(S, i, S->n[1] + NG, k)] = 0.0;
        }
      }
  }
  if (S->bc[0][0] == BC_OUTFLOW || S->bc[0][1] == BC_OUTFLOW) {
    for (int k = NG - 1; k <= S->n[2] + NG; k++)
      for (int j = NG - 1; j <= S->n[1] + NG; j++) {
        if (S->bc[0][0] == BC_OUTFLOW) {
          long id = IDX(S, NG, j, k);
          if (S->F[0][RHO * N + id] > 0.0) {
            S->F[0][RHO * N + id] = 0.0;
            if (S->elec)
              for (int q = 0; q < 2; q++) S->FK[0][q * N + id] = 0.0;
          }
        }
        if (S->bc[0][1] == BC_OUTFLOW) {
          long id = IDX(S, S->n[0] + NG, j, k);
          if (S->F[0][RHO * N + id] < 0.0) {
            S->F[0][RHO * N + id] = 0.0;
            if (S->elec)
              for (int q = 0; q < 2; q++) S->FK[0][q * N + id] = 0.0;
          }
        }
      }
  }
}

/* Flux-CT (Toth 2000): corner EMFs as the average of the four face fluxes
 * that meet at an edge, then every induction flux is replaced by the
 * average of the two EMFs bounding its face.  F_d[B_d] = 0. */
static void flux_ct(Sim *S) {
  const long N = S->ntot;
  const int n1 = S->n[0], n2 = S->n[1], n3 = S->n[2];
  std::vector<real> &F1 = S->F[0], &F2 = S->F[1], &F3 = S->F[2];
  std::vector<real> &e1 = S->emf[0], &e2 = S->emf[1], &e3 = S->emf[2];
  for (int k = NG; k <= n3 + NG; k++)
    for (int j = NG; j <= n2 + NG; j++)
      for (int i = NG; i <= n1 + NG; i++) {
        long c = IDX(S, i, j, k);
        long im = IDX(S, i - 1, j, k), jm = IDX(S, i, j - 1, k), km = IDX(S, i, j, k - 1);
        e3[c] = 0.25 * (F1[B2 * N + c] + F1[B2 * N + jm] - F2[B1 * N + c] - F2[B1 * N + im]);
        e2[c] = 0.25 * (F3[B1 * N + c] + F3[B1 * N + im] - F1[B3 * N + c] - F1[B3 * N + km]);
        e1[c] = 0.25 * (F2[B3 * N + c] + F2[B3 * N + km] - F3[B2 * N + c] - F3[B2 * N + jm]);
      }
  /* X1 faces */
  for (int k = NG; k < n3 + NG; k++)
    for (int j = NG; j < n2 + NG; j++)
      for (int i = NG; i <= n1 + NG; i++) {
        long c = IDX(S, i, j, k);
        F1[B1 * N + c] = 0.0;
        F1[B2 * N + c] = 0.5 * (e3[c] + e3[IDX(S, i, j + 1, k)]);
        F1[B3 * N + c] = -0.5 * (e2[c] + e2[IDX(S, i, j, k + 1)]);
      }
  /* X2 faces */
  for (int k = NG; k < n3 + NG; k++)
    for (int j = NG; j <= n2 + NG; j++)
      for (int i = NG; i < n1 + NG; i++) {
        long c = IDX(S, i, j, k);
        F2[B1 * N + c] = -0.5 * (e3[c] + e3[IDX(S, i + 1, j, k)]);
        F2[B2 * N + c] = 0.0;
        F2[B3 * N + c] = 0.5 * (e1[c] + e1[IDX(S, i, j, k + 1)]);
      }
  /* X3 faces */
  for (int k = NG; k <= n3 + NG; k++)
    for (int j = NG; j < n2 + NG; j++)
      for (int i = NG; i < n1 + NG; i++) {
        long c = IDX(S, i, j, k);
        F3[B1 * N + c] = 0.5 * (e2[c] + e2[IDX(S, i + 1, j, k)]);
        F3[B2 * N + c] = -0.5 * (e1[c] + e1[IDX(S, i, j + 1, k)]);
        F3[B3 * N + c] = 0.0;
      }
}

/* ------------------------------------------------------------------------ */
/* Geometric source sqrt(-g) T^kappa_lambda Gamma^lambda_{nu kappa}            */
/* ------------------------------------------------------------------------ */
static void fluid_source(const real P[NPRIM], const FluidState &s, const GeomPt &g,
                         const real *conn, real gam, real dU[NPRIM]) {
  real T[4][4];
  for (int mu = 0; mu < 4; mu++) mhd_row(P, s, gam, mu, T[mu]);
  for (int v = 0; v < NPRIM; v++) dU[v] = 0.0;
  for (int nu = 0; nu < 4; nu++) {
    real acc = 0.0;
    for (int ka = 0; ka < 4; ka++)
      for (int la = 0; la < 4; la++) acc += T[ka][la] * conn[(la * 4 + nu) * 4 + ka];
    dU[UU + nu] = acc * g.gdet;
  }
}

/* ------------------------------------------------------------------------ */
/* 1D_W primitive recovery (Noble et al. 2006), solved for W' = W - D.        */
/* ------------------------------------------------------------------------ */
struct InvInput {
  real D, Qpn, Qtsq, QdB, Bsq;
};

static real vsq_of_W(const InvInput &q, real W) {
  real W2 = W * W;
  real BW = q.Bsq + W;
  return (q.Qtsq * W2 + q.QdB * q.QdB * (q.Bsq + 2.0 * W)) / (BW * BW * W2);
}

static real dvsq_dW(const InvInput &q, real W) {
  real W3 = W * W * W;
  real BW = q.Bsq + W;
  return -2.0 * (q.Qtsq * W3 + q.QdB * q.QdB * (3.0 * W * W + 3.0 * W * q.Bsq + q.Bsq * q.Bsq)) /
         (BW * BW * BW * W3);
}

/* w - rho = W (1-v^2) - D sqrt(1-v^2), written without the cancellation of
 * the rest mass: W'(1-v^2) - D v^2 sqrt(1-v^2)/(1+sqrt(1-v^2)). */
static real w_minus_rho(const InvInput &q, real Wp, real vsq) {
  real sq = rsqrt_(1.0 - vsq);
  return Wp * (1.0 - vsq) - q.D * vsq * sq / (1.0 + sq);
}

static int u_to_p(const real U[NPRIM], const GeomPt &g, real gam, const real Pg[NPRIM],
                  real P[NPRIM]) {
  for (int v = 0; v < NPRIM; v++) P[v] = Pg[v];
  real gdet = g.gdet, alpha = g.alpha;
  /* primitive field B^i = U_B/sqrt(-g); normal-observer field is alpha B^i */
  real Bp[4] = {0.0, U[B1] / gdet, U[B2] / gdet, U[B3] / gdet};
  P[B1] = Bp[1];
  P[B2] = Bp[2];
  P[B3] = Bp[3];
  InvInput q;
  q.D = U[RHO] * alpha / gdet;
  if (!(q.D > 0.0)) return INV_D_NEG;
  real Bn[4] = {0.0, alpha * Bp[1], alpha * Bp[2], alpha * Bp[3]};
  /* Q_mu = alpha T^t_mu (rest mass restored in Q_t) */
  real Qcov[4];
  Qcov[0] = alpha * (U[UU] - U[RHO]) / gdet;
  for (int i = 1; i < 4; i++) Qcov[i] = alpha * U[UU + i] / gdet;
  /* n^mu = -alpha g^{mu t};  Q'.n = Q.n + D without the rest-mass cancellation:
   * Q_t n^t = (U_E - U_rho)/sqrt(-g), D = alpha U_rho/sqrt(-g). */
  real Qpn = (U[UU] - (1.0 - alpha) * U[RHO]) / gdet;
  for (int i = 1; i < 4; i++) Qpn += Qcov[i] * (-alpha * g.gcon[i][0]);
  q.Qpn = Qpn;
  /* projected Q: Qtilde^i = gamma^{ij} Q_j, gamma^{ij} = g^{ij} - g^{it} g^{jt}/g^{tt} */
  real Qt[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = 1; i < 4; i++)
    for (int j = 1; j < 4; j++)
      Qt[i] += (g.gcon[i][j] - g.gcon[i][0] * g.gcon[j][0] / g.gcon[0][0]) * Qcov[j];
  q.Qtsq = 0.0;
  for (int i = 1; i < 4; i++) q.Qtsq += Qt[i] * Qcov[i];
  q.QdB = 0.0;
  for (int i = 1; i < 4; i++) q.QdB += Qcov[i] * Bn[i];
  q.Bsq = 0.0;
  for (int i = 1; i < 4; i++)
    for (int j = 1; j < 4; j++) q.Bsq += g.gcov[i][j] * Bn[i] * Bn[j];

  /* guess W' from the guess primitives */
  real qsq = 0.0;
  for (int i = 1; i < 4; i++)
    for (int j = 1; j < 4; j++) qsq += g.gcov[i][j] * Pg[U1 + i - 1] * Pg[U1 + j - 1];
  real gsq = 1.0 + qsq;
  /* rho + u + p = rho + gamma_ad u.  A physical state has W = (rho + gamma_ad u)
   * gamma^2 >= rho gamma = D, i.e. W' >= 0: the guess is clamped there. */
  real Wp = (Pg[RHO] + gam * Pg[UU]) * gsq - q.D;
  if (Wp < 0.0) Wp = 0.0;

  const real gfac = (gam - 1.0) / gam;
  int converged = 0, extra = 0, invalid = 0, have_hi = 0;
  real lo = 0.0, hi = 0.0; /* bracket on W' from the sign of f and from v^2 >= 1 */
  for (int it = 0; it < INV_MAXIT + INV_EXTRA; it++) {
    real W = Wp + q.D;
    real vsq = vsq_of_W(q, W);
    invalid = 0;
    if (vsq > INV_VSQ_MAX) {
      /* v^2(W) decreases with W: this iterate lies below the root. */
      lo = rmax(lo, Wp);
      Wp = have_hi ? 0.5 * (lo + hi) : Wp + W;
      invalid = 1;
      if (converged || it + 1 >= INV_MAXIT) break;
      continue;
    }
    if (vsq < 0.0) vsq = 0.0;
    real pr = gfac * w_minus_rho(q, Wp, vsq);
    real f = q.Qpn + Wp - pr + 0.5 * (1.0 + vsq) * q.Bsq - 0.5 * q.QdB * q.QdB / (W * W);
    if (f > 0.0) {
      hi = have_hi ? rmin(hi, Wp) : Wp;
      have_hi = 1;
    } else {
      lo = rmax(lo, Wp);
    }
    real dv = dvsq_dW(q, W);
    real sq = rsqrt_(1.0 - vsq);
    real dpdW = gfac * ((1.0 - vsq) + dv * (0.5 * q.D / sq - W));
    real df = 1.0 - dpdW + 0.5 * q.Bsq * dv + q.QdB * q.QdB / (W * W * W);
    real Wn = Wp - f / df;
    if (Wn < 0.0) Wn = 0.5 * Wp;
    if (converged) {
      Wp = Wn;
      extra++;
      if (extra >= INV_EXTRA) break;
      continue;
    }
    if (rabs(Wn - Wp) <= INV_TOL * rabs(W)) converged = 1;
    Wp = Wn;
    if (!converged && it + 1 >= INV_MAXIT) break;
  }
  real W = Wp + q.D;
  if (!converged) return INV_NOCONV;
  if (!(W > 0.0) || !rfinite(W)) return INV_W_BAD;
  real vsq = vsq_of_W(q, W);
  if (!(vsq < 1.0) || invalid) return INV_VSQ;
  if (vsq < 0.0) vsq = 0.0;
  real sq = rsqrt_(1.0 - vsq);
  real rho = q.D * sq;
  real uu = w_minus_rho(q, Wp, vsq) / gam;
  if (!(rho > 0.0)) return INV_RHO_NEG;
  if (uu < 0.0) return INV_U_NEG;
  real gamma = 1.0 / sq;
  real fac = gamma / (W + q.Bsq);
  P[RHO] = rho;
  P[UU] = uu;
  for (int i = 1; i < 4; i++) P[U1 + i - 1] = fac * (Qt[i] + q.QdB * Bn[i] / W);
  return INV_OK;
}

/* ------------------------------------------------------------------------ */
/* Floors (paper, "Implementation Notes", bounds list; no electron bound).    */
/* READING: the Lorentz-factor cap is applied first (it changes b^2), then    */
/* rho and u are raised in the fluid frame in the listed order, so every      */
/* bound holds at once on exit.                                              */
/* ------------------------------------------------------------------------ */
static int apply_floors(real P[NPRIM], const GeomPt &g, real rho_fl, real u_fl, real gam) {
  int flags = 0;
  real qsq = 0.0;
  for (int i = 1; i < 4; i++)
    for (int j = 1; j < 4; j++) qsq += g.gcov[i][j] * P[U1 + i - 1] * P[U1 + j - 1];
  real gamma = rsqrt_(1.0 + qsq);
  if (gamma > GAMMA_MAX) {
    real f = rsqrt_((GAMMA_MAX * GAMMA_MAX - 1.0) / qsq);
    for (int i = 0; i < 3; i++) P[U1 + i] *= f;
    flags |= FF_GAMMA;
  }
  FluidState s;
  get_state(P, g, s);
  if (P[RHO] < rho_fl) { P[RHO] = rho_fl; flags |= FF_RHO_GEOM; }
  if (P[UU] < u_fl) { P[UU] = u_fl; flags |= FF_U_GEOM; }
  real rmin_sig = s.bsq / BSQ_OVER_RHO_MAX;
  if (P[RHO] < rmin_sig) { P[RHO] = rmin_sig; flags |= FF_SIGMA; }
  real umin_beta = BETA_MIN * s.bsq / (2.0 * (gam - 1.0));
  if (P[UU] < umin_beta) { P[UU] = umin_beta; flags |= FF_BETA; }
  real rmin_t = P[UU] / U_OVER_RHO_MAX;
  if (P[RHO] < rmin_t) { P[RHO] = rmin_t; flags |= FF_TEMP; }
  return flags;
}

/* ------------------------------------------------------------------------ */
/* READING (drift-frame bounds; a variant the paper's bounds list leaves      */
/* open).  The mass and internal energy that the fluid-frame bounds would     */
/* add are added instead as a field-free parcel that moves with the zone's    */
/* drift velocity: the part of the fluid 3-velocity seen by the normal        */
/* observer that is perpendicular to B (the E x B drift of ideal MHD), so     */
/* that floor material brings no momentum along the field.  With v = u~/gam  */
/* (gam = sqrt(1 + u~.u~)) and B-hat = B/|B| in the spatial metric g_ij, the  */
/* drift velocity is v_d = v - (v.B-hat) B-hat, its Lorentz factor is         */
/* gam/sqrt(1 + (u~.B-hat)^2), hence u~_d = (u~ - (u~.B-hat) B-hat) /        */
/* sqrt(1 + (u~.B-hat)^2).  The direction of a field too weak to matter is   */
/* set by rounding, so a field with g_ij B^i B^j <= 1e-20 rho (rho after the  */
/* bounds) counts as none: the parcel then moves with the fluid.  The         */
/* parcel's conserved variables are added to U(P) (P after the Lorentz-factor */
/* cap) and the sum is inverted by 1D_W from the fluid-frame result; the      */
/* fluid-frame bounds are then applied once more, so every bound holds on     */
/* exit.  Where B = 0 or v is perpendicular to B the parcel moves with the    */
/* fluid and the result is the fluid-frame one up to the inversion's          */
/* round-off.  If the inversion fails, the fluid-frame result is kept.        */
/* Ppre (may be NULL) receives the inverted state before that last pass.      */
/* ------------------------------------------------------------------------ */
static int apply_floors_drift(real P[NPRIM], const GeomPt &g, real rho_fl, real u_fl, real gam,
                              real *Ppre) {
  real Pf[NPRIM];
  for (int v = 0; v < NPRIM; v++) Pf[v] = P[v];
  int flags = apply_floors(Pf, g, rho_fl, u_fl, gam);
  if (!(flags & ~FF_GAMMA)) {
    for (int v = 0; v < NPRIM; v++) P[v] = Pf[v];
    return flags;
  }
  /* the state the bounds act on: P's rho and u, the (capped) velocity */
  real Pc[NPRIM];
  for (int v = 0; v < NPRIM; v++) Pc[v] = P[v];
  for (int i = 0; i < 3; i++) Pc[U1 + i] = Pf[U1 + i];
  real Pp[NPRIM];
  Pp[RHO] = Pf[RHO] - Pc[RHO];
  Pp[UU] = Pf[UU] - Pc[UU];
  real udB = 0.0, Bsq = 0.0;
  for (int i = 1; i < 4; i++)
    for (int j = 1; j < 4; j++) {
      udB += g.gcov[i][j] * Pc[U1 + i - 1] * Pc[B1 + j - 1];
      Bsq += g.gcov[i][j] * Pc[B1 + i - 1] * Pc[B1 + j - 1];
    }
  if (Bsq > DRIFT_BSQ_MIN * Pf[RHO]) {
    real upar2 = udB * udB / Bsq; /* (u~.B-hat)^2 */
    real f = 1.0 / rsqrt_(1.0 + upar2);
    for (int i = 0; i < 3; i++) Pp[U1 + i] = f * (Pc[U1 + i] - (udB / Bsq) * Pc[B1 + i]);
  } else {
    for (int i = 0; i < 3; i++) Pp[U1 + i] = Pc[U1 + i];
  }
  Pp[B1] = Pp[B2] = Pp[B3] = 0.0;
  FluidState sc, sp;
  get_state(Pc, g, sc);
  get_state(Pp, g, sp);
  real Uc[NPRIM], Up[NPRIM], Us[NPRIM];
  prim_to_flux(Pc, sc, g, gam, 0, Uc);
  prim_to_flux(Pp, sp, g, gam, 0, Up);
  for (int v = 0; v < NPRIM; v++) Us[v] = Uc[v] + Up[v];
  real Pn[NPRIM];
  int pf = u_to_p(Us, g, gam, Pf, Pn);
  if (pf != INV_OK) {
    for (int v = 0; v < NPRIM; v++) P[v] = Pf[v];
    return flags | FF_DRIFT_FAIL;
  }
  if (Ppre)
    for (int v = 0; v < NPRIM; v++) Ppre[v] = Pn[v];
  flags |= FF_DRIFT | apply_floors(Pn, g, rho_fl, u_fl, gam);
  for (int v = 0; v < NPRIM; v++) P[v] = Pn[v];
  return flags;
}

/* ------------------------------------------------------------------------ */
/* Electron heating fraction f_e, the share of the dissipated internal       */
/* energy that goes to the electrons, from a zone's rho, u, b^2 and          */
/* kappa_e.  Temperatures (units of m_p c^2): u_e = kappa_e                   */
/* rho^gamma_e/(gamma_e - 1), T_e = (gamma_e - 1) u_e/rho, T_p = (gamma_p -   */
/* 1)(u - u_e)/rho; the proton beta is beta_p = rho T_p/(b^2/2).             */
/* READING: temperatures enter by magnitude, T_p/T_e is clamped to          */
/* [1e-20, 1e20] and beta_p to [1e-20, 1e20] (1e20: an unmagnetised zone).  */
/* Each model is the fit its paper publishes, with f_e = 1/(1 + Q_i/Q_e):     */
/*  Kawazura et al. 2019  Q_i/Q_e = 35/(1 + (beta_p/15)^-1.4 e^(-0.1 T_e/T_p)) */
/*  Werner et al. 2018    f_e = (1 + sqrt((s/5)/(2 + s/5)))/4, s = b^2/rho    */
/*  Rowan et al. 2017     f_e = exp(-(1 - beta_p/beta_max)^3.3 /              */
/*                        (1 + 1.2 s_w^0.7))/2, s_w = b^2/(rho + u + p),      */
/*                        beta_max = 1/(4 s_w), beta_p capped at beta_max     */
/*  Sharma et al. 2007    Q_e/Q_i = 0.33 sqrt(T_e/T_p)                        */
/*  Howes 2010            Q_i/Q_e = c1 (c2^2 + beta_p^x)/(c3^2 + beta_p^x)    */
/*                        sqrt(m_p T_p/(m_e T_e)) e^(-1/beta_p), x = 2 -      */
/*                        0.2 log10(T_p/T_e), c1 = 0.92; c2 = 1.6 T_e/T_p and */
/*                        c3 = 18 + 5 log10(T_p/T_e) for T_p > T_e, else      */
/*                        c2 = 1.2 T_e/T_p, c3 = 18                           */
/* ------------------------------------------------------------------------ */
static real elec_fraction(const ElecParams &e, real rho, real u, real kel, real bsq) {
  if (e.model == ELEC_CONSTANT) return e.fel_const;
  real ue = kel * rpow(rho, e.game) / (e.game - 1.0);
  real Te = rabs((e.game - 1.0) * ue / rho);
  real Tp = rabs((e.gamp - 1.0) * (u - ue) / rho);
  real trat = (Te > 0.0) ? Tp / Te : real(ELEC_BETA_CAP); /* T_p / T_e */
  trat = rmin(rmax(trat, real(1.0e-20)), real(1.0e20));
  real beta = (bsq > 0.0) ? 2.0 * rho * Tp / bsq : real(ELEC_BETA_CAP);
  beta = rmin(rmax(beta, real(1.0 / ELEC_BETA_CAP)), real(ELEC_BETA_CAP));
  if (e.model == ELEC_KAWAZURA) {
    real qiqe = 35.0 / (1.0 + rpow(beta / 15.0, -1.4) * rexp(-0.1 / trat));
    return 1.0 / (1.0 + qiqe);
  }
  if (e.model == ELEC_WERNER) {
    real s = bsq / rho;
    return 0.25 * (1.0 + rsqrt_((s / 5.0) / (2.0 + s / 5.0)));
  }
  if (e.model == ELEC_ROWAN) {
    real sw = bsq / (rho + e.gam * u);
    real r = rmin(4.0 * sw * beta, real(1.0)); /* beta_p / beta_max */
    return 0.5 * rexp(-rpow(1.0 - r, 3.3) / (1.0 + 1.2 * rpow(sw, 0.7)));
  }
  if (e.model == ELEC_SHARMA) {
    real qeqi = 0.33 * rsqrt_(1.0 / trat);
    return qeqi / (1.0 + qeqi);
  }
  if (e.model == ELEC_HOWES) {
    real lt = rlog10(trat);
    real c2 = (trat > 1.0) ? 1.6 / trat : 1.2 / trat;
    real c3 = (trat > 1.0) ? 18.0 + 5.0 * lt : real(18.0);
    real bx = rpow(beta, 2.0 - 0.2 * lt);
    real qiqe = 0.92 * (c2 * c2 + bx) / (c3 * c3 + bx) * rsqrt_(MP_OVER_ME * trat) *
                rexp(-1.0 / beta);
    return 1.0 / (1.0 + qiqe);
  }
  return 0.0;
}

/* Electron heating (Ressler et al. 2015) of one zone after its inversion.
 * kappa_tot_new = (gamma - 1) u/rho^gamma of the updated state is the
 * entropy the fluid has; kappa_tot,adv, carried without dissipation, the
 * entropy it would have had; the electrons take the share f_e of the
 * difference, as internal energy at the density rho_s:
 *   kappa_e = kappa_e,adv + f_e (gamma_e - 1)/(gamma - 1) rho_s^(gamma - gamma_e)
 *             (kappa_tot_new - kappa_tot,adv),
 * i.e. rho_s^gamma_e d(kappa_e)/(gamma_e - 1) = f_e rho_s^gamma d(kappa_tot)/(gamma - 1).
 * READING: rho_s and f_e come from the stage's source state (the state the
 * geometric source uses), and the heating precedes the bounds, so that
 * floor material brings the electrons no heat. */
static real elec_heat(const ElecParams &e, real rho_s, real fel, real ktot_new, real ktot_adv,
                      real kel_adv) {
  return kel_adv + fel * (e.game - 1.0) / (e.gam - 1.0) * rpow(rho_s, e.gam - e.game) *
                       (ktot_new - ktot_adv);
}

/* Bounds on kappa_e from T_p/T_e in [tpte_min, tpte_max]: with p_e = rho T_e,
 * p_p = rho T_p and u = p_e/(gamma_e - 1) + p_p/(gamma_p - 1) = p/(gamma - 1),
 * a ratio R = T_p/T_e gives kappa_e = kappa_tot rho^(gamma - gamma_e) /
 * ((gamma - 1)/(gamma_e - 1) + R (gamma - 1)/(gamma_p - 1)).  A kappa_e that
 * is not a number takes the lower bound. */
static real elec_bound(const ElecParams &e, real rho, real ktot, real kel) {
  real a = (e.gam - 1.0) / (e.game - 1.0), b = (e.gam - 1.0) / (e.gamp - 1.0);
  real kk = ktot * rpow(rho, e.gam - e.game);
  real kmax = kk / (a + e.tpte_min * b);
  real kmin = kk / (a + e.tpte_max * b);
  if (!(kel == kel)) kel = kmin;
  return rmin(rmax(kel, kmin), kmax);
}

/* The closing steps of a zone's electron state once the fluid's bounds are
 * done: u lowered so that P_gas/rho^gamma <= 3 (paper, bounds list, when
 * electron temperatures are evolved; with the bounds on), kappa_tot reset to
 * the state's, kappa_e bounded.  Returns FF_KTOT if u was lowered. */
static int elec_close(const Sim *S, real P[NPRIM], real K[2]) {
  const ElecParams &e = S->ep;
  int fl = 0;
  if (S->floors_on) {
    real kt = (e.gam - 1.0) * P[UU] / rpow(P[RHO], e.gam);
    if (kt > KTOT_MAX) {
      P[UU] = KTOT_MAX * rpow(P[RHO], e.gam) / (e.gam - 1.0);
      fl = FF_KTOT;
    }
  }
  K[0] = (e.gam - 1.0) * P[UU] / rpow(P[RHO], e.gam);
  K[1] = elec_bound(e, P[RHO], K[0], K[1]);
  return fl;
}

/* ------------------------------------------------------------------------ */
/* One stage: U(Pi) + dt'[-div F + S(Ps)] -> invert -> floors -> fixup.      */
/* ------------------------------------------------------------------------ */
/* Ki, Ks, Kout: the electron entropies of the same stage arrays (empty
 * without electrons; Kout may be Ki, each zone reads its own first). */
static int advance_stage(Sim *S, const std::vector<real> &Pi, const std::vector<real> &Ps,
                         std::vector<real> &Pout, double dtp, const std::vector<real> &Ki,
                         const std::vector<real> &Ks, std::vector<real> &Kout) {
  const long N = S->ntot;
  const int n1 = S->n[0], n2 = S->n[1], n3 = S->n[2];
  bool same = (&Pi == &Ps);
  /* update + inversion + floors */
  for (int k = NG; k < n3 + NG; k++)
    for (int j = NG; j < n2 + NG; j++)
      for (int i = NG; i < n1 + NG; i++) {
        long c = IDX(S, i, j, k);
        long ij = IJ(S, i, j);
        const GeomPt &g = S->geom[LOC_CENT][ij];
        real pi[NPRIM], ps[NPRIM], Ui[NPRIM], dU[NPRIM], Unew[NPRIM], pn[NPRIM];
        load_prims(S, Pi, c, pi);
        FluidState si, ss;
        get_state(pi, g, si);
        prim_to_flux(pi, si, g, S->gam, 0, Ui);
        if (same) {
          fluid_source(pi, si, g, &S->conn[ij * 64], S->gam, dU);
        } else {
          load_prims(S, Ps, c, ps);
          get_state(ps, g, ss);
          fluid_source(ps, ss, g, &S->conn[ij * 64], S->gam, dU);
        }
        long cp1 = IDX(S, i + 1, j, k), cp2 = IDX(S, i, j + 1, k), cp3 = IDX(S, i, j, k + 1);
        for (int v = 0; v < NPRIM; v++) {
          real div = (S->F[0][v * N + cp1] - S->F[0][v * N + c]) / S->dx[0] +
                     (S->F[1][v * N + cp2] - S->F[1][v * N + c]) / S->dx[1] +
                     (S->F[2][v * N + cp3] - S->F[2][v * N + c]) / S->dx[2];
          Unew[v] = Ui[v] + dtp * (dU[v] - div);
        }
        int pf = u_to_p(Unew, g, S->gam, pi, pn);
        int ff = 0;
        real kn[2] = {0.0, 0.0};
        if (S->elec) {
          /* the entropies carried with the mass: U_K = sqrt(-g) rho u^t K */
          real kadv[2];
          for (int q = 0; q < 2; q++) {
            long o = (long)q * N;
            real divk = (S->FK[0][o + cp1] - S->FK[0][o + c]) / S->dx[0] +
                        (S->FK[1][o + cp2] - S->FK[1][o + c]) / S->dx[1] +
                        (S->FK[2][o + cp3] - S->FK[2][o + c]) / S->dx[2];
            real Uk = Ui[RHO] * Ki[o + c] + dtp * (0.0 - divk);
            kadv[q] = Uk / Unew[RHO];
          }
          kn[0] = kadv[0];
          kn[1] = kadv[1];
          if (pf == INV_OK) {
            const real *psrc = same ? pi : ps;
            FluidState st;
            get_state(psrc, g, st);
            real fel = elec_fraction(S->ep, psrc[RHO], psrc[UU], Ks[N + c], st.bsq);
            real ktot_new = (S->gam - 1.0) * pn[UU] / rpow(pn[RHO], S->gam);
            kn[1] = elec_heat(S->ep, psrc[RHO], fel, ktot_new, kadv[0], kadv[1]);
            if (S->floors_on)
              ff = (S->floor_frame == FLOOR_DRIFT)
                       ? apply_floors_drift(pn, g, S->rho_floor[ij], S->u_floor[ij], S->gam, nullptr)
                       : apply_floors(pn, g, S->rho_floor[ij], S->u_floor[ij], S->gam);
            ff |= elec_close(S, pn, kn);
          }
        } else if (pf == INV_OK && S->floors_on) {
          ff = (S->floor_frame == FLOOR_DRIFT)
                   ? apply_floors_drift(pn, g, S->rho_floor[ij], S->u_floor[ij], S->gam, nullptr)
                   : apply_floors(pn, g, S->rho_floor[ij], S->u_floor[ij], S->gam);
        }
        S->pflag[c] = pf;
        S->fflag[c] = ff;
        for (int v = 0; v < NPRIM; v++) Pout[v * N + c] = pn[v];
        if (S->elec)
          for (int q = 0; q < 2; q++) Kout[(long)q * N + c] = kn[q];
      }
  /* fixup of failed zones: mean of the non-failed interior zones of the
   * 3x3x3 neighbourhood (rho, u, utilde); B is kept.  READING.  The bounds
   * of a fixed-up zone are the fluid-frame ones in either frame: the
   * neighbour mean it takes conserves nothing to begin with. */
#ifdef ORACLE_COUNT
  int saved_phase = g_phase;
  g_phase = 3;
#endif
  int unrecoverable = 0;
  for (int k = NG; k < n3 + NG; k++)
    for (int j = NG; j < n2 + NG; j++)
      for (int i = NG; i < n1 + NG; i++) {
        long c = IDX(S, i, j, k);
        if (S->pflag[c] == INV_OK) continue;
        S->inv_fail_total++;
        real sum[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, sumk = 0.0;
        int cnt = 0;
        for (int dk = -1; dk <= 1; dk++)
          for (int dj = -1; dj <= 1; dj++)
            for (int di = -1; di <= 1; di++) {
              if (di == 0 && dj == 0 && dk == 0) continue;
              int ii = i + di, jj = j + dj, kk = k + dk;
              if (ii < NG || ii >= n1 + NG || jj < NG || jj >= n2 + NG || kk < NG || kk >= n3 + NG)
                continue;
              long nb = IDX(S, ii, jj, kk);
              if (S->pflag[nb] != INV_OK) continue;
              for (int v = 0; v < 5; v++) sum[v] += Pout[v * N + nb];
              if (S->elec) sumk += Kout[N + nb];
              cnt++;
            }
        if (cnt == 0) {
          unrecoverable++;
          continue; /* keeps the guess values; reported as an error */
        }
        real pn[NPRIM];
        load_prims(S, Pout, c, pn);
        for (int v = 0; v < 5; v++) pn[v] = sum[v] / (double)cnt;
        long ij = IJ(S, i, j);
        if (S->floors_on)
          S->fflag[c] |= apply_floors(pn, S->geom[LOC_CENT][ij], S->rho_floor[ij], S->u_floor[ij], S->gam);
        if (S->elec) {
          /* READING: kappa_e takes the same neighbour mean; kappa_tot follows u */
          real kn[2] = {0.0, sumk / (double)cnt};
          S->fflag[c] |= elec_close(S, pn, kn);
          for (int q = 0; q < 2; q++) Kout[(long)q * N + c] = kn[q];
        }
        for (int v = 0; v < NPRIM; v++) Pout[v * N + c] = pn[v];
      }
  for (int k = NG; k < n3 + NG; k++)
    for (int j = NG; j < n2 + NG; j++)
      for (int i = NG; i < n1 + NG; i++)
        if (S->fflag[IDX(S, i, j, k)]) S->floor_hits_total++;
  S->unrecoverable_total += unrecoverable;
#ifdef ORACLE_COUNT
  g_phase = saved_phase;
#endif
  bounds(S, Pout, Kout);
  return unrecoverable;
}

/* READING (time step): ndt_d = CFL dX_d / max_faces ctop_d over the interior
 * faces of each direction with more than one zone; dt = 1/sum_d(1/ndt_d);
 * dt <= 1.3 dt_previous; the last step lands on t_final.  dt comes from the
 * fluxes of the state at the start of the step (the predictor's fluxes). */
static double compute_dt(Sim *S) {
  double inv = 0.0;
  for (int d = 0; d < 3; d++) {
    if (S->n[d] <= 1) continue;
    double ct = val(S->ctop_max[d]);
    if (ct > 0.0) {
      double ndt = S->cfl * S->dx[d] / ct;
      inv += 1.0 / ndt;
    }
  }
  double dt = (inv > 0.0) ? 1.0 / inv : INFINITY;
  if (S->dt_prev > 0.0 && dt > 1.3 * S->dt_prev) dt = 1.3 * S->dt_prev;
  if (S->t_final > 0.0 && S->t + dt > S->t_final) dt = S->t_final - S->t;
  if (!(dt > 0.0)) dt = 0.0;
  return dt;
}

#ifdef ORACLE_COUNT
#define PHASE(p) (g_phase = (p))
#else
#define PHASE(p) ((void)0)
#endif

static int step_once(Sim *S) {
  /* predictor: Ps = Pi = P^n, dt' = dt/2 -> Ph */
  PHASE(0);
  get_fluxes(S, S->P, S->K);
  PHASE(4);
  double dt = compute_dt(S);
  if (!std::isfinite(dt)) return -3;
  if (dt <= 0.0) return 0; /* at t_final: the step is a no-op */
  PHASE(1);
  fix_flux(S);
  flux_ct(S);
  PHASE(2);
  int bad = advance_stage(S, S->P, S->P, S->Ph, 0.5 * dt, S->K, S->K, S->Kh);
  /* corrector: Ps = P^{n+1/2}, Pi = P^n, dt' = dt -> P^{n+1} */
  PHASE(0);
  get_fluxes(S, S->Ph, S->Kh);
  PHASE(1);
  fix_flux(S);
  flux_ct(S);
  PHASE(2);
  bad += advance_stage(S, S->P, S->Ph, S->P, dt, S->K, S->Kh, S->K);
  PHASE(4);
  S->t += dt;
  S->dt = dt;
  S->dt_prev = dt;
  S->nstep++;
  return bad ? -4 : 0;
}

/* ------------------------------------------------------------------------ */
/* C ABI for ctypes                                                          */
/* ------------------------------------------------------------------------ */
extern "C" {

void *oracle_create(const int n[3], const double xmin[3], const double xmax[3], int metric,
                    double a, double hslope, double gam, double cfl, double t_final, int recon,
                    int floors_on, const int bc[6]) {
  Sim *S = new Sim();
  for (int d = 0; d < 3; d++) {
    S->n[d] = n[d];
    S->s[d] = n[d] + 2 * NG;
    S->xmin[d] = xmin[d];
    S->xmax[d] = xmax[d];
    S->dx[d] = (xmax[d] - xmin[d]) / n[d];
    S->bc[d][0] = bc[2 * d];
    S->bc[d][1] = bc[2 * d + 1];
  }
  S->ntot = (long)S->s[0] * S->s[1] * S->s[2];
  S->metric = metric;
  S->a = a;
  S->hslope = hslope;
  S->gam = gam;
  S->cfl = cfl;
  S->t_final = t_final;
  S->recon = recon;
  S->floors_on = floors_on;
  S->floor_frame = FLOOR_FLUID;
  S->elec = ELEC_OFF;
  S->ep = ElecParams{ELEC_OFF, gam, 0.0, 0.0, 0.0, 0.0, 0.0};
  build_geometry(S);
  S->P.assign(NPRIM * S->ntot, real(0.0));
  S->Ph.assign(NPRIM * S->ntot, real(0.0));
  S->Lz.assign(NPRIM * S->ntot, real(0.0));
  S->Rz.assign(NPRIM * S->ntot, real(0.0));
  for (int d = 0; d < 3; d++) {
    S->F[d].assign(NPRIM * S->ntot, real(0.0));
    S->emf[d].assign(S->ntot, real(0.0));
  }
  S->pflag.assign(S->ntot, 0);
  S->fflag.assign(S->ntot, 0);
  S->t = 0.0;
  S->dt = 0.0;
  S->dt_prev = 0.0;
  S->nstep = 0;
  S->inv_fail_total = S->floor_hits_total = S->unrecoverable_total = 0;
  return S;
}

void oracle_destroy(void *h) { delete (Sim *)h; }

/* frame of the bounds: FLOOR_FLUID (default) or FLOOR_DRIFT */
void oracle_set_floor_frame(void *h, int frame) { ((Sim *)h)->floor_frame = frame; }

/* Evolve the electron entropies with heating model `model` (ELEC_*; 0
 * turns them off).  Call before setting the state; kappa starts at 0. */
void oracle_set_electrons(void *h, int model, double game, double gamp, double fel_const,
                          double tpte_min, double tpte_max) {
  Sim *S = (Sim *)h;
  S->elec = model;
  S->ep.model = model;
  S->ep.gam = S->gam;
  S->ep.game = game;
  S->ep.gamp = gamp;
  S->ep.fel_const = fel_const;
  S->ep.tpte_min = tpte_min;
  S->ep.tpte_max = tpte_max;
  if (model) {
    S->K.assign(2 * S->ntot, real(0.0));
    S->Kh.assign(2 * S->ntot, real(0.0));
    S->KLz.assign(2 * S->ntot, real(0.0));
    S->KRz.assign(2 * S->ntot, real(0.0));
    for (int d = 0; d < 3; d++) S->FK[d].assign(2 * S->ntot, real(0.0));
  } else {
    S->K.clear();
    S->Kh.clear();
    for (int d = 0; d < 3; d++) S->FK[d].clear();
  }
}

/* K: (kappa_tot, kappa_e) as [2][n3][n2][n1] (with_ghosts = 0) or
 * [2][s3][s2][s1]; ghosts are then filled by the BCs as for the primitives
 * (which are filled again, unchanged). */
void oracle_set_K(void *h, const double *K, int with_ghosts) {
  Sim *S = (Sim *)h;
  if (!S->elec) return;
  if (with_ghosts) {
    for (long q = 0; q < 2 * S->ntot; q++) S->K[q] = K[q];
  } else {
    for (int v = 0; v < 2; v++)
      for (int k = 0; k < S->n[2]; k++)
        for (int j = 0; j < S->n[1]; j++)
          for (int i = 0; i < S->n[0]; i++)
            S->K[v * S->ntot + IDX(S, i + NG, j + NG, k + NG)] =
                K[(((long)v * S->n[2] + k) * S->n[1] + j) * S->n[0] + i];
  }
  bounds(S, S->P, S->K);
  S->Ph = S->P;
  S->Kh = S->K;
}

void oracle_get_K(void *h, double *K, int with_ghosts) {
  Sim *S = (Sim *)h;
  if (!S->elec) return;
  if (with_ghosts) {
    for (long q = 0; q < 2 * S->ntot; q++) K[q] = val(S->K[q]);
    return;
  }
  for (int v = 0; v < 2; v++)
    for (int k = 0; k < S->n[2]; k++)
      for (int j = 0; j < S->n[1]; j++)
        for (int i = 0; i < S->n[0]; i++)
          K[(((long)v * S->n[2] + k) * S->n[1] + j) * S->n[0] + i] =
              val(S->K[v * S->ntot + IDX(S, i + NG, j + NG, k + NG)]);
}

/* pointwise: the heating fraction of a zone, and one heating update */
double oracle_elec_fraction(int model, double gam, double game, double gamp, double fel_const,
                            double rho, double u, double kel, double bsq) {
  ElecParams e = {model, gam, game, gamp, fel_const, 0.0, 0.0};
  return val(elec_fraction(e, rho, u, kel, bsq));
}

double oracle_elec_heat(double gam, double game, double rho_s, double fel, double ktot_new,
                        double ktot_adv, double kel_adv) {
  ElecParams e = {ELEC_CONSTANT, gam, game, 0.0, fel, 0.0, 0.0};
  return val(elec_heat(e, rho_s, fel, ktot_new, ktot_adv, kel_adv));
}

/* P: [8][n3][n2][n1] interior primitives; ghosts are filled by the BCs
 * (BC_FIXED ghosts are left as they are). */
/* READING (fixed boundaries): the ghosts of a BC_FIXED side hold their set
 * values in both stage arrays, so the half-step state starts as a copy. */
void oracle_set_prims(void *h, const double *P) {
  Sim *S = (Sim *)h;
  for (int v = 0; v < NPRIM; v++)
    for (int k = 0; k < S->n[2]; k++)
      for (int j = 0; j < S->n[1]; j++)
        for (int i = 0; i < S->n[0]; i++)
          S->P[v * S->ntot + IDX(S, i + NG, j + NG, k + NG)] =
              P[(((long)v * S->n[2] + k) * S->n[1] + j) * S->n[0] + i];
  bounds(S, S->P, S->K);
  S->Ph = S->P;
  S->Kh = S->K;
}

/* P: [8][s3][s2][s1] including ghosts; then the BCs are applied. */
void oracle_set_prims_ghost(void *h, const double *P) {
  Sim *S = (Sim *)h;
  for (long q = 0; q < NPRIM * S->ntot; q++) S->P[q] = P[q];
  bounds(S, S->P, S->K);
  S->Ph = S->P;
  S->Kh = S->K;
}

void oracle_get_prims(void *h, double *P, int with_ghosts) {
  Sim *S = (Sim *)h;
  if (with_ghosts) {
    for (long q = 0; q < NPRIM * S->ntot; q++) P[q] = val(S->P[q]);
    return;
  }
  for (int v = 0; v < NPRIM; v++)
    for (int k = 0; k < S->n[2]; k++)
      for (int j = 0; j < S->n[1]; j++)
        for (int i = 0; i < S->n[0]; i++)
          P[(((long)v * S->n[2] + k) * S->n[1] + j) * S->n[0] + i] =
              val(S->P[v * S->ntot + IDX(S, i + NG, j + NG, k + NG)]);
}

/* Advance nsteps full predictor-corrector steps (fewer once t reaches a
 * positive t_final).  Returns 0, -3 (no finite dt) or -4 (a failed zone had
 * no valid neighbour in some stage). */
int oracle_step(void *h, int nsteps) {
  Sim *S = (Sim *)h;
  int rc = 0;
  for (int s = 0; s < nsteps; s++) {
    if (S->t_final > 0.0 && S->t >= S->t_final) break; /* nothing left to do */
    int r = step_once(S);
    if (r != 0) rc = r;
    if (r == -3) break;
  }
  return rc;
}

/* The predictor stage alone: P <- P^{n+1/2} (t is not advanced).  Returns
 * the number of unrecoverable zones. */
int oracle_predictor(void *h) {
  Sim *S = (Sim *)h;
  get_fluxes(S, S->P, S->K);
  double dt = compute_dt(S);
  if (!(dt > 0.0) || !std::isfinite(dt)) return -3;
  fix_flux(S);
  flux_ct(S);
  int bad = advance_stage(S, S->P, S->P, S->Ph, 0.5 * dt, S->K, S->K, S->Kh);
  S->P.swap(S->Ph);
  S->K.swap(S->Kh);
  return bad;
}

void oracle_get_time(void *h, double out[3]) {
  Sim *S = (Sim *)h;
  out[0] = S->t;
  out[1] = S->dt;
  out[2] = (double)S->nstep;
}

/* Restore the clock of a checkpoint: time t and the previous step's dt
 * (the growth limit of the next step depends on it). */
void oracle_set_time(void *h, double t, double dt_prev, long nstep) {
  Sim *S = (Sim *)h;
  S->t = t;
  S->dt = dt_prev;
  S->dt_prev = dt_prev;
  S->nstep = nstep;
}

void oracle_get_counters(void *h, long out[3]) {
  Sim *S = (Sim *)h;
  out[0] = S->inv_fail_total;
  out[1] = S->floor_hits_total;
  out[2] = S->unrecoverable_total;
}

/* pflag/fflag of the last stage, interior [n3][n2][n1] */
void oracle_get_flags(void *h, int *pflag, int *fflag) {
  Sim *S = (Sim *)h;
  for (int k = 0; k < S->n[2]; k++)
    for (int j = 0; j < S->n[1]; j++)
      for (int i = 0; i < S->n[0]; i++) {
        long o = ((long)k * S->n[1] + j) * S->n[0] + i;
        long c = IDX(S, i + NG, j + NG, k + NG);
        pflag[o] = S->pflag[c];
        fflag[o] = S->fflag[c];
      }
}

/* Fluxes of the current state after the boundary fixes and flux-CT,
 * F: [3][8][s3][s2][s1]; ctop: max ctop per direction over interior faces. */
void oracle_get_fluxes(void *h, double *F, double ctop[3]) {
  Sim *S = (Sim *)h;
  get_fluxes(S, S->P, S->K);
  fix_flux(S);
  flux_ct(S);
  for (int d = 0; d < 3; d++) {
    for (long q = 0; q < NPRIM * S->ntot; q++) F[d * NPRIM * S->ntot + q] = val(S->F[d][q]);
    ctop[d] = val(S->ctop_max[d]);
  }
}

/* The dt the next step would take (from the fluxes of the current state). */
double oracle_next_dt(void *h) {
  Sim *S = (Sim *)h;
  get_fluxes(S, S->P, S->K);
  return compute_dt(S);
}

/* Geometry at location loc (0 CENT, 1 FACE1, 2 FACE2), 2D [s2][s1] arrays,
 * packed as out[comp][s2][s1] with comp = gcov(16), gcon(16), gdet, alpha;
 * and conn (64 components) at CENT when loc == 3. */
void oracle_get_geom(void *h, int loc, double *out) {
  Sim *S = (Sim *)h;
  long n2d = (long)S->s[0] * S->s[1];
  for (long q = 0; q < n2d; q++) {
    if (loc == 3) {
      for (int c = 0; c < 64; c++) out[c * n2d + q] = val(S->conn[q * 64 + c]);
      continue;
    }
    const GeomPt &G = S->geom[loc][q];
    for (int m = 0; m < 4; m++)
      for (int n = 0; n < 4; n++) {
        out[(m * 4 + n) * n2d + q] = val(G.gcov[m][n]);
        out[(16 + m * 4 + n) * n2d + q] = val(G.gcon[m][n]);
      }
    out[32 * n2d + q] = val(G.gdet);
    out[33 * n2d + q] = val(G.alpha);
  }
}

/* ---- pointwise entry points for the pins ---- */
static void geom_from_point(int kind, double a, double h, const double X[4], GeomPt &G) {
  double gcov[4][4], gcon[4][4], gd, al;
  geom_point(kind, a, h, X, gcov, gcon, &gd, &al);
  for (int m = 0; m < 4; m++)
    for (int n = 0; n < 4; n++) { G.gcov[m][n] = gcov[m][n]; G.gcon[m][n] = gcon[m][n]; }
  G.gdet = gd;
  G.alpha = al;
}

/* gcov(16), gcon(16), gdet, alpha, conn(64) at X */
void oracle_geom_at(int kind, double a, double h, const double X[4], double *out) {
  double gcov[4][4], gcon[4][4], gd, al, cn[4][4][4];
  geom_point(kind, a, h, X, gcov, gcon, &gd, &al);
  conn_point(kind, a, h, X, cn);
  for (int q = 0; q < 16; q++) { out[q] = (&gcov[0][0])[q]; out[16 + q] = (&gcon[0][0])[q]; }
  out[32] = gd;
  out[33] = al;
  for (int q = 0; q < 64; q++) out[34 + q] = (&cn[0][0][0])[q];
}

/* U (dir 0) or F (dir 1..3) of P at X */
void oracle_prim_to_flux(int kind, double a, double h, const double X[4], double gam,
                         const double *P, int dir, double *F) {
  GeomPt G;
  geom_from_point(kind, a, h, X, G);
  real p[NPRIM], f[NPRIM];
  for (int v = 0; v < NPRIM; v++) p[v] = P[v];
  FluidState s;
  get_state(p, G, s);
  prim_to_flux(p, s, G, gam, dir, f);
  for (int v = 0; v < NPRIM; v++) F[v] = val(f[v]);
}

/* b^2 and u^mu, b^mu of P at X: out = bsq, ucon[4], bcon[4] */
void oracle_state_at(int kind, double a, double h, const double X[4], const double *P,
                     double *out) {
  GeomPt G;
  geom_from_point(kind, a, h, X, G);
  real p[NPRIM];
  for (int v = 0; v < NPRIM; v++) p[v] = P[v];
  FluidState s;
  get_state(p, G, s);
  out[0] = val(s.bsq);
  for (int m = 0; m < 4; m++) { out[1 + m] = val(s.ucon[m]); out[5 + m] = val(s.bcon[m]); }
}

int oracle_cons_to_prim(int kind, double a, double h, const double X[4], double gam,
                        const double *U, const double *Pguess, double *P) {
  GeomPt G;
  geom_from_point(kind, a, h, X, G);
  real u[NPRIM], pg[NPRIM], p[NPRIM];
  for (int v = 0; v < NPRIM; v++) { u[v] = U[v]; pg[v] = Pguess[v]; }
  int rc = u_to_p(u, G, gam, pg, p);
  for (int v = 0; v < NPRIM; v++) P[v] = val(p[v]);
  return rc;
}

void oracle_vchar(int kind, double a, double h, const double X[4], double gam, const double *P,
                  int dir, double out[2]) {
  GeomPt G;
  geom_from_point(kind, a, h, X, G);
  real p[NPRIM];
  for (int v = 0; v < NPRIM; v++) p[v] = P[v];
  FluidState s;
  get_state(p, G, s);
  real vmax, vmin;
  vchar(p, s, G, gam, dir, &vmax, &vmin);
  out[0] = val(vmax);
  out[1] = val(vmin);
}

/* geometric source sqrt(-g) T^k_l Gamma^l_{nu k} at X (8 entries) */
void oracle_source_at(int kind, double a, double h, const double X[4], double gam,
                      const double *P, double *dU) {
  GeomPt G;
  geom_from_point(kind, a, h, X, G);
  double cn[4][4][4];
  conn_point(kind, a, h, X, cn);
  real c[64], p[NPRIM], d[NPRIM];
  for (int q = 0; q < 64; q++) c[q] = (&cn[0][0][0])[q];
  for (int v = 0; v < NPRIM; v++) p[v] = P[v];
  FluidState s;
  get_state(p, G, s);
  fluid_source(p, s, G, c, gam, d);
  for (int v = 0; v < NPRIM; v++) dU[v] = val(d[v]);
}

int oracle_floors_at(int kind, double a, double h, const double X[4], double gam, double *P) {
  GeomPt G;
  geom_from_point(kind, a, h, X, G);
  double r = std::exp(X[1]);
  double kk = 1.0 / (r * r * (1.0 + r / 10.0));
  real p[NPRIM];
  for (int v = 0; v < NPRIM; v++) p[v] = P[v];
  int fl = apply_floors(p, G, FLOOR_RHO_K * kk, FLOOR_U_K * std::pow(kk, gam), gam);
  for (int v = 0; v < NPRIM; v++) P[v] = val(p[v]);
  return fl;
}

/* the drift-frame bounds at one point; Ppre (8 doubles, may be NULL): the
 * inverted state before the closing fluid-frame pass (untouched unless
 * FF_DRIFT is set) */
int oracle_floors_drift_at(int kind, double a, double h, const double X[4], double gam, double *P,
                           double *Ppre) {
  GeomPt G;
  geom_from_point(kind, a, h, X, G);
  double r = std::exp(X[1]);
  double kk = 1.0 / (r * r * (1.0 + r / 10.0));
  real p[NPRIM], pre[NPRIM];
  for (int v = 0; v < NPRIM; v++) p[v] = P[v];
  for (int v = 0; v < NPRIM; v++) pre[v] = 0.0;
  int fl = apply_floors_drift(p, G, FLOOR_RHO_K * kk, FLOOR_U_K * std::pow(kk, gam), gam, pre);
  for (int v = 0; v < NPRIM; v++) P[v] = val(p[v]);
  if (Ppre && (fl & FF_DRIFT))
    for (int v = 0; v < NPRIM; v++) Ppre[v] = val(pre[v]);
  return fl;
}

/* the step's reconstruction of one zone: out = (low face, high face) */
void oracle_recon(int kind, const double *x, double out[2]) {
  real l, r;
  if (kind == RECON_WENO5) {
    real xx[5];
    for (int q = 0; q < 5; q++) xx[q] = x[q];
    weno5_zone(xx, &l, &r);
  } else {
    recon_mc(x[0], x[1], x[2], &l, &r);
  }
  out[0] = val(l);
  out[1] = val(r);
}

/* the single-face textbook form: out = (low face, high face), each from
 * its own indicators */
void oracle_recon_faces(const double *x, double out[2]) {
  real xx[5], l, r;
  for (int q = 0; q < 5; q++) xx[q] = x[q];
  recon_weno5(xx, &l, &r);
  out[0] = val(l);
  out[1] = val(r);
}

int oracle_is_counting(void) {
#ifdef ORACLE_COUNT
  return 1;
#else
  return 0;
#endif
}

/* add/sub, mul, div, sqrt counts per phase since the last reset, out[6][4]
 * (phases: face fluxes, flux fixes + flux-CT, update + inversion + floors,
 * fixup, other, reconstruction); zeros in the plain build. */
void oracle_op_counts(double out[24], int reset) {
#ifdef ORACLE_COUNT
  for (int p = 0; p < 6; p++) {
    out[4 * p + 0] = g_phase_ops[p].add;
    out[4 * p + 1] = g_phase_ops[p].mul;
    out[4 * p + 2] = g_phase_ops[p].div;
    out[4 * p + 3] = g_phase_ops[p].sqrt;
    if (reset) g_phase_ops[p] = OpCounts{0, 0, 0, 0};
  }
#else
  (void)reset;
  for (int q = 0; q < 24; q++) out[q] = 0.0;
#endif
}

} /* extern "C" */
