// grmhd_dev.cuh -- device-side data layout and per-point physics of the
// GB300 GRMHD step (HARM scheme as implemented by iharm3D, arXiv:2110.10191).
//
// Layout (HBM): every zone-centred or face-centred field is a
// structure-of-arrays of float64, field[v][k][j][i] with i fastest and 3 ghost
// layers per side.  Face arrays use the index of the zone whose low face
// they sit on (face i-1/2 of zone i).  Geometry is X3-independent (both
// supported metrics are), so it lives in 2D [comp][j][i] arrays that stay
// resident in L2 for the whole step.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace grmhd {

constexpr int NV = 8;
constexpr int NG = 3;
enum { RHO = 0, UU, U1, U2, U3, B1, B2, B3 };

// Packed symmetric 4x4 index: (0,0)0 (0,1)1 (0,2)2 (0,3)3 (1,1)4 (1,2)5
// (1,3)6 (2,2)7 (2,3)8 (3,3)9.
__host__ __device__ constexpr int SY(int m, int n) {
  return (m <= n) ? (m * 4 - (m * (m - 1)) / 2 + (n - m)) : (n * 4 - (n * (n - 1)) / 2 + (m - n));
}

// geometry components of one location
constexpr int G_GCOV = 0;    // 10 packed g_{mu nu}
constexpr int G_GCON = 10;   // 10 packed g^{mu nu}
constexpr int G_GDET = 20;   // sqrt(-g)
constexpr int G_ALPHA = 21;  // lapse 1/sqrt(-g^{tt})
constexpr int G_IALPHA = 22; // 1/lapse
constexpr int G_IGDET = 23;  // 1/sqrt(-g)
constexpr int G_OMALPHA = 24; // 1 - lapse, formed in FP64 (for the FP32 energy flux)
constexpr int G_NCOMP = 25;
constexpr int C_NCOMP = 40;  // connection Gamma^l_{(m n)}: l*10 + SY(m,n)
enum { LOC_CENT = 0, LOC_FACE1 = 1, LOC_FACE2 = 2, NLOC = 3 };

// bound constants (paper, "Implementation Notes", list of bounds)
constexpr double FL_RHO_K = 1.0e-6;
constexpr double FL_U_K = 1.0e-8;
constexpr double FL_SIGMA = 400.0;
constexpr double FL_BETA = 2.5e-5;
constexpr double FL_TEMP = 100.0;
constexpr double FL_GAMMA = 50.0;
constexpr double FL_DRIFT_BSQ = 1.0e-20;  // drift-frame bounds: weaker fields count as none
// correctly rounded reciprocals of the divisors above
constexpr double FL_SIGMA_RCP = 1.0 / FL_SIGMA;
constexpr double FL_TEMP_RCP = 1.0 / FL_TEMP;

// Adiabatic-index constants of the inversion and the bounds, formed once on
// the host: gamma, 1/gamma, (gamma - 1)/gamma, and the beta bound's divisor
// 2 (gamma - 1) with its correctly rounded reciprocal.
struct GasK {
  double gam, igam, gf, ubd, ubd_rcp;
};
enum {
  FF_GAMMA = 1, FF_RHO_GEOM = 2, FF_U_GEOM = 4, FF_SIGMA = 8, FF_BETA = 16, FF_TEMP = 32,
  FF_DRIFT = 64,      // drift-frame bounds: parcel added, sum inverted
  FF_DRIFT_FAIL = 128 // that inversion failed: the fluid-frame result was kept
};
enum { PF_OK = 0, PF_NOCONV = 1, PF_W = 2, PF_VSQ = 3, PF_RHO = 4, PF_U = 5, PF_D = 6 };

// Reciprocal without the IEEE division sequence: the hardware approximation
// (PTX rcp.approx.ftz.f64, about 20 correct bits) refined by one third-order
// step of the geometric series 1/x = r/(1 - e) = r (1 + e + e^2 + ...),
// e = 1 - x r: r <- r + r (e + e^2), which leaves a relative error of about
// e^3 ~ 2^-60 before the final rounding (three FMAs; two Newton-Raphson
// steps, r <- r + r e twice, take four for the same result).  Within a few
// ulp of 1/x for normal x.  Used where the quotient feeds further arithmetic
// (WENO weights, signal speeds, the Newton iteration of the inversion);
// decisions compared against constants keep IEEE division.
__device__ __forceinline__ double rcp_nr(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
}

// Reciprocal square root without the IEEE sequence: the hardware
// approximation (PTX rsqrt.approx.ftz.f64) refined by the binomial series
// (1 - h)^(-1/2) = 1 + h/2 + 3h^2/8 + ... with h = 1 - x y^2, y the seed:
// y <- y + y h (1/2 + 3h/8), which leaves about (5/16) h^3 of the seed's
// relative error h before the final rounding (five FP64 instructions).
// Within a few ulp of 1/sqrt(x) for normal positive x.
__device__ __forceinline__ double rsqrt_nr(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double h = fma(-(x * y), y, 1.0);
  return fma(y * h, fma(0.375, h, 0.5), y);
}

// Square root of a positive normal x as x / sqrt(x) from rsqrt_nr (within a
// few ulp); the callers send zero, negative and subnormal values to their
// own branch.
__device__ __forceinline__ double sqrt_nr(double x) { return x * rsqrt_nr(x); }

// smallest positive normal double
constexpr double DBL_NORMAL_MIN = 2.2250738585072014e-308;

// x / c correctly rounded, from rc = RN(1/c): q0 = x rc is within one ulp of
// x/c, its residual x - q0 c is exact in one FMA, and q0 + r rc rounds to
// RN(x/c) (Markstein's correction, IBM J. Res. Dev. 34 (1990) 111).  For
// finite x with x/c and x rc in the normal range; three FP64 instructions
// where the IEEE division sequence takes several more.
__device__ __forceinline__ double div_rn(double x, double c, double rc) {
  const double q0 = x * rc;
  const double r = fma(-q0, c, x);
  return fma(r, rc, q0);
}

struct Dims {
  int n[3];   // interior zones
  int s[3];   // with ghosts
  long long ntot;
  long long n2d;  // s[0]*s[1]
};

__device__ __forceinline__ long long zid(const Dims &D, int i, int j, int k) {
  return ((long long)k * D.s[1] + j) * D.s[0] + i;
}

struct Geo {
  double gcov[10], gcon[10], gdet, alpha, ialpha, igdet;
};

__device__ __forceinline__ void load_geo(const double *__restrict__ g, long long n2d, long long ij,
                                         Geo &G) {
#pragma unroll
  for (int c = 0; c < 10; c++) G.gcov[c] = __ldg(g + (G_GCOV + c) * n2d + ij);
#pragma unroll
  for (int c = 0; c < 10; c++) G.gcon[c] = __ldg(g + (G_GCON + c) * n2d + ij);
  G.gdet = __ldg(g + G_GDET * n2d + ij);
  G.alpha = __ldg(g + G_ALPHA * n2d + ij);
  G.ialpha = __ldg(g + G_IALPHA * n2d + ij);
  G.igdet = __ldg(g + G_IGDET * n2d + ij);
}

// ---------------------------------------------------------------------------
// Fluid state u^mu, u_mu, b^mu, b_mu, b^2 of one primitive vector.
// u^t = gamma/alpha, u^i = utilde^i - gamma alpha g^{ti}; u_i = g_ij utilde^j,
// u_t = -alpha gamma + g_tj utilde^j (the normal observer has n_i = 0);
// b^t = B^i u_i, b^i = (B^i + b^t u^i)/u^t.
// ---------------------------------------------------------------------------
struct FState {
  double ucon[4], ucov[4], bcon[4], bcov[4], bsq;
};

__device__ __forceinline__ void fluid_state(const double P[NV], const Geo &G, FState &s) {
  const double v1 = P[U1], v2 = P[U2], v3 = P[U3];
  const double l1 = G.gcov[SY(1, 1)] * v1 + G.gcov[SY(1, 2)] * v2 + G.gcov[SY(1, 3)] * v3;
  const double l2 = G.gcov[SY(1, 2)] * v1 + G.gcov[SY(2, 2)] * v2 + G.gcov[SY(2, 3)] * v3;
  const double l3 = G.gcov[SY(1, 3)] * v1 + G.gcov[SY(2, 3)] * v2 + G.gcov[SY(3, 3)] * v3;
  // gamma and 1/gamma from one reciprocal square root
  const double g2 = fma(l1, v1, fma(l2, v2, fma(l3, v3, 1.0)));
  const double rg = rsqrt_nr(g2);
  const double gam = g2 * rg;
  const double ga = gam * G.alpha;
  s.ucon[0] = gam * G.ialpha;
  s.ucon[1] = v1 - ga * G.gcon[SY(0, 1)];
  s.ucon[2] = v2 - ga * G.gcon[SY(0, 2)];
  s.ucon[3] = v3 - ga * G.gcon[SY(0, 3)];
  s.ucov[0] = fma(G.gcov[SY(0, 1)], v1, fma(G.gcov[SY(0, 2)], v2, fma(G.gcov[SY(0, 3)], v3, -ga)));
  s.ucov[1] = l1;
  s.ucov[2] = l2;
  s.ucov[3] = l3;
  const double bt = P[B1] * l1 + P[B2] * l2 + P[B3] * l3;
  const double iut = G.alpha * rg;  // 1/u^t
  s.bcon[0] = bt;
  s.bcon[1] = (P[B1] + bt * s.ucon[1]) * iut;
  s.bcon[2] = (P[B2] + bt * s.ucon[2]) * iut;
  s.bcon[3] = (P[B3] + bt * s.ucon[3]) * iut;
#pragma unroll
  for (int m = 0; m < 4; m++) {
    double a = 0.0;
#pragma unroll
    for (int n = 0; n < 4; n++) a += G.gcov[SY(m, n)] * s.bcon[n];
    s.bcov[m] = a;
  }
  s.bsq = s.bcon[0] * s.bcov[0] + s.bcon[1] * s.bcov[1] + s.bcon[2] * s.bcov[2] +
          s.bcon[3] * s.bcov[3];
}

// sqrt(-g)-weighted conserved densities (dir 0) or fluxes (dir 1..3):
// rho u^d ; T^d_t + rho u^d ; T^d_i ; b^j u^d - b^d u^j, with
// T^d_nu = (rho + u + p + b^2) u^d u_nu + (p + b^2/2) delta^d_nu - b^d b_nu.
__device__ __forceinline__ void prim_flux(const double P[NV], const FState &s, const Geo &G,
                                          double gam, int dir, double F[NV]) {
  const double pg = (gam - 1.0) * P[UU];
  const double w = P[RHO] + P[UU] + pg + s.bsq;
  const double pt = pg + 0.5 * s.bsq;
  const double wu = w * s.ucon[dir];
  const double bd = s.bcon[dir];
  double T[4];
#pragma unroll
  for (int nu = 0; nu < 4; nu++) T[nu] = wu * s.ucov[nu] - bd * s.bcov[nu];
  T[dir] += pt;
  const double mflux = P[RHO] * s.ucon[dir];
  F[RHO] = G.gdet * mflux;
  F[UU] = G.gdet * (T[0] + mflux);
  F[U1] = G.gdet * T[1];
  F[U2] = G.gdet * T[2];
  F[U3] = G.gdet * T[3];
  const double ud = s.ucon[dir];
  F[B1] = G.gdet * (s.bcon[1] * ud - bd * s.ucon[1]);
  F[B2] = G.gdet * (s.bcon[2] * ud - bd * s.ucon[2]);
  F[B3] = G.gdet * (s.bcon[3] * ud - bd * s.ucon[3]);
}

// acc (+)= F^dir + coef * U without the sqrt(-g) factor: the two rows
// T^dir_nu and T^t_nu share (rho + u + p + b^2) u_nu and b_nu.  FIRST: acc
// is set rather than added to (the first state of a face).  gm1 = gamma - 1.
template <bool FIRST>
__device__ __forceinline__ void flux_cons_acc(const double P[NV], const FState &s, double gm1,
                                              int dir, double coef, double acc[NV]) {
  const double pg = gm1 * P[UU];
  const double w = P[RHO] + P[UU] + pg + s.bsq;
  const double pt = pg + 0.5 * s.bsq;
  const double ud = s.ucon[dir], ut = s.ucon[0];
  const double bd = s.bcon[dir], bt = s.bcon[0];
  // combined contravariant weights: F + coef U = (u^d + coef u^t) ... - (b^d + coef b^t) ...
  const double uc = ud + coef * ut;
  const double bc = bd + coef * bt;
  const double wuc = w * uc;
  double T[4];
#pragma unroll
  for (int nu = 0; nu < 4; nu++) T[nu] = wuc * s.ucov[nu] - bc * s.bcov[nu];
  T[dir] += pt;
  T[0] += coef * pt;
  const double mf = P[RHO] * uc;
  const double add[NV] = {mf,
                          T[0] + mf,
                          T[1],
                          T[2],
                          T[3],
                          s.bcon[1] * uc - bc * s.ucon[1],
                          s.bcon[2] * uc - bc * s.ucon[2],
                          s.bcon[3] * uc - bc * s.ucon[3]};
#pragma unroll
  for (int v = 0; v < NV; v++) acc[v] = FIRST ? add[v] : acc[v] + add[v];
}

// Fast-magnetosonic coordinate speeds along dir: roots v of
// (k.u)^2 = cms2 (k.k + (k.u)^2) for k_mu = delta^dir_mu - v delta^t_mu,
// cms2 = cs2 + va2 - cs2 va2; a negative discriminant counts as zero.
// With cs2 = gamma (gamma - 1) u / e_f, va2 = b^2 / (b^2 + e_f) and
// e_f = rho + gamma u, the combination is exactly
// cms2 = (gamma (gamma - 1) u + b^2) / (b^2 + e_f): one reciprocal, no
// cancellation.  ggm1 = gamma (gamma - 1).  Returns the larger magnitude of
// the two roots (hb +- disc)/qa, disc >= 0: (|hb| + disc)/|qa|, the same
// rounded value as the larger rounded root's magnitude (the LLF flux and
// the time step need only it).
__device__ __forceinline__ double mhd_cmax(const double P[NV], const FState &s, const Geo &G,
                                           double gam, double ggm1, int dir) {
  const double ef = fma(gam, P[UU], P[RHO]);
  const double ee = s.bsq + ef;
  const double cms2 = fma(ggm1, P[UU], s.bsq) * rcp_nr(ee);
  const double Asq = G.gcon[SY(dir, dir)];
  const double Bsq = G.gcon[SY(0, 0)];
  const double AB = G.gcon[SY(0, dir)];
  const double Au = s.ucon[dir];
  const double Bu = s.ucon[0];
  const double AuBu = Au * Bu;
  // qa v^2 - 2 hb v + qc = 0: roots (hb +- sqrt(hb^2 - qa qc)) / qa
  const double qa = Bu * Bu - (Bsq + Bu * Bu) * cms2;
  const double hb = AuBu - (AB + AuBu) * cms2;
  const double qc = Au * Au - (Asq + Au * Au) * cms2;
  double disc = fma(hb, hb, -(qa * qc));
  disc = (disc >= DBL_NORMAL_MIN) ? sqrt_nr(disc) : 0.0;  // a subnormal root is negligible
  return (fabs(hb) + disc) * fabs(rcp_nr(qa));
}

// ---------------------------------------------------------------------------
// Reconstruction
// ---------------------------------------------------------------------------
// MC limited slope of x1 with neighbours x0, x2.
__device__ __forceinline__ double mc_slope(double x0, double x1, double x2) {
  const double dm = x1 - x0, dp = x2 - x1;
  if (!(dm * dp > 0.0)) return 0.0;
  const double dc = 0.5 * (dm + dp);
  const double m = fmin(fmin(fabs(2.0 * dm), fabs(dc)), fabs(2.0 * dp));
  return (dc > 0.0) ? m : -m;
}

// Jiang-Shu WENO5 value at the high face of the middle zone of a..e
// (cell averages; epsilon 1e-26, weights d_k/(eps + beta_k)^2).
__device__ __forceinline__ double weno5_hi(double a, double b, double c, double d, double e) {
  const double eps = 1.0e-26;
  const double t0 = a - 2.0 * b + c, t1 = b - 2.0 * c + d, t2 = c - 2.0 * d + e;
  const double s0 = a - 4.0 * b + 3.0 * c, s1 = b - d, s2 = 3.0 * c - 4.0 * d + e;
  const double b0 = (13.0 / 12.0) * t0 * t0 + 0.25 * s0 * s0;
  const double b1 = (13.0 / 12.0) * t1 * t1 + 0.25 * s1 * s1;
  const double b2 = (13.0 / 12.0) * t2 * t2 + 0.25 * s2 * s2;
  const double e0 = eps + b0, e1 = eps + b1, e2 = eps + b2;
  const double q0 = e0 * e0, q1 = e1 * e1, q2 = e2 * e2;
  // alpha_k = d_k / q_k ; common denominator q0 q1 q2
  const double a0 = 0.1 * (q1 * q2), a1 = 0.6 * (q0 * q2), a2 = 0.3 * (q0 * q1);
  const double p0 = (2.0 * a - 7.0 * b + 11.0 * c) * (1.0 / 6.0);
  const double p1 = (-b + 5.0 * c + 2.0 * d) * (1.0 / 6.0);
  const double p2 = (2.0 * c + 5.0 * d - e) * (1.0 / 6.0);
  return (a0 * p0 + a1 * p1 + a2 * p2) / (a0 + a1 + a2);
}

// Both WENO5 face values of the middle zone of a..e (zones c-2..c+2), written
// in the stencil's first differences (dm2 = b-a, dm1 = c-b, dp1 = d-c,
// dp2 = e-d), second differences (D0 = a-2b+c, D1 = b-2c+d, D2 = c-2d+e) and
// s0 = D0 + 2 dm1, s1 = dm1 + dp1, s2 = D2 - 2 dp1:
//   4 beta_k = (13/3) D_k^2 + s_k^2,
// and, with q_k the candidate values at the high face,
//   6 (q_0 - c) = A = 2 D0 + 3 dm1 = Cl + D0,   Cl = D0 + 3 dm1 = s0 + dm1,
//   6 (q_1 - c) = B = dm1 + 2 dp1  = s1 + dp1,
//   6 (q_2 - c) = C = 3 dp1 - D2   = dp1 - s2,
// the low face's by mirroring: Al = 2 D2 - 3 dp1 = D2 - C, Bl = dp1 + 2 dm1
// = s1 + dm1, Cl.  The weights d_k/(eps + beta_k)^2 are taken over the
// common denominator q0 q1 q2 of the squared (4 eps + 4 beta_k) and scaled
// by 10, which leaves their ratios unchanged, and one reciprocal serves
// both faces, with the 1/6 of the candidate differences folded into it.
// 4 eps + 4 beta_k = s_k^2 + T_k with T_k = (13/3) D_k^2 + 4 eps, a
// function of the one second difference D_k: along a column the T_k of
// one zone are T_{k+1}, T_{k+2} of its lower neighbours, so a walk forms one
// new D and T per zone (weno5_walk).  The terms pair up under the mirror
// a <-> e, b <-> d (A <-> Al, B <-> -Bl, C <-> -Cl, D0 <-> D2, s0 <-> -s2),
// so a mirrored stencil gives the same two values swapped, bit for bit.
__device__ __forceinline__ double weno5_T(double Dk) {
  return fma((13.0 / 3.0) * Dk, Dk, 4.0e-26);
}

__device__ __forceinline__ void weno5_pair_dt(double c, double dm1, double dp1, double D0,
                                              double D1, double D2, double T0, double T1,
                                              double T2, double &lo, double &hi) {
  const double s0 = fma(2.0, dm1, D0), s1 = dm1 + dp1, s2 = fma(-2.0, dp1, D2);
  const double e0 = fma(s0, s0, T0), e1 = fma(s1, s1, T1), e2 = fma(s2, s2, T2);
  const double q0 = e0 * e0, q1 = e1 * e1, q2 = e2 * e2;
  // linear weights in the ratio 1 : 6 : 3 (only ratios enter)
  const double q12 = q1 * q2, q02 = 6.0 * (q0 * q2), q01 = q0 * q1;
  const double t01 = 3.0 * q01, t12 = 3.0 * q12;
  const double Cl = s0 + dm1, A = Cl + D0, B = s1 + dp1, C = dp1 - s2;
  const double Al = D2 - C, Bl = s1 + dm1;
  // high face: weights q12, 6 q02, 3 q01
  const double nh = fma(t01, C, fma(q02, B, q12 * A));
  const double H = (q12 + q02) + t01;
  // low face (mirrored stencil): weights q01, 6 q02, 3 q12
  const double nl = fma(-t12, Cl, fma(-q02, Bl, q01 * Al));
  const double L = (q01 + q02) + t12;
  const double r = rcp_nr(H * L) * (1.0 / 6.0);
  hi = fma(nh, L * r, c);
  lo = fma(nl, H * r, c);
}

__device__ __forceinline__ void weno5_pair(double a, double b, double c, double d, double e,
                                           double &lo, double &hi) {
  const double dm2 = b - a, dm1 = c - b, dp1 = d - c, dp2 = e - d;
  const double D0 = dm1 - dm2, D1 = dp1 - dm1, D2 = dp2 - dp1;
  weno5_pair_dt(c, dm1, dp1, D0, D1, D2, weno5_T(D0), weno5_T(D1), weno5_T(D2), lo, hi);
}

// Both face values of n <= 16 consecutive zones of one column (stride st;
// p, lf and rf point at the first zone): each zone after the first loads one
// new value and forms one first difference, one second difference and one
// T_k; the values equal weno5_pair's on each zone's stencil bit for bit.
__device__ __forceinline__ void weno5_walk(const double *__restrict__ p, double *__restrict__ lf,
                                           double *__restrict__ rf, long long st, int n) {
  const double xm1 = __ldg(p - st);
  double x0 = __ldg(p), xp1 = __ldg(p + st), xp2 = __ldg(p + 2 * st);
  double dm1 = x0 - xm1, dp1 = xp1 - x0, dp2 = xp2 - xp1;
  double D0 = dm1 - (xm1 - __ldg(p - 2 * st)), D1 = dp1 - dm1, D2 = dp2 - dp1;
  double T0 = weno5_T(D0), T1 = weno5_T(D1), T2 = weno5_T(D2);
  // unrolled over the longest segment (the segments' length is at most 16):
  // a rolled loop of unknown trip count ran 12% slower
#pragma unroll
  for (int m = 0; m < 16; m++) {
    // the next zone's new value, loaded before this zone's arithmetic
    const double xn = (m + 1 < n) ? __ldg(p + (m + 3) * st) : 0.0;
    double lo, hi;
    weno5_pair_dt(x0, dm1, dp1, D0, D1, D2, T0, T1, T2, lo, hi);
    lf[m * st] = lo;
    rf[m * st] = hi;
    if (m + 1 >= n) break;
    const double dn = xn - xp2;
    x0 = xp1;
    xp1 = xp2;
    xp2 = xn;
    dm1 = dp1;
    dp1 = dp2;
    D0 = D1;
    D1 = D2;
    D2 = dn - dp2;
    dp2 = dn;
    T0 = T1;
    T1 = T2;
    T2 = weno5_T(D2);
  }
}

// ---------------------------------------------------------------------------
// 1D_W primitive recovery (Noble et al. 2006) in W' = W - D.
// Iteration rule: guess W' from the guess primitives (clamped >= 0); Newton
// until a step <= 1e-8 W, then 1 more step (round-off by quadratic
// convergence); at most 16 (+1) iterations; a
// step below W' = 0 halves W'; an iterate with v^2 > 1 - 1e-10 is replaced by
// the bisection of the bracket known from sign(f), or doubles W while no
// upper end is known.
// ---------------------------------------------------------------------------
constexpr int INV_MAXIT = 16;
constexpr int INV_EXTRA = 1;
constexpr double INV_TOL = 1.0e-8;
constexpr double INV_VSQ_MAX = 1.0 - 1.0e-10;

// On success also returns b^2 = B^2 (1 - v^2) + (Q.B / W)^2 (normal-frame
// field B, B.v = Q.B/W) and the Lorentz factor of the recovered state, so the
// bounds need not rebuild the fluid state.
__device__ __forceinline__ int invert_1dw(const double U[NV], const Geo &G, const GasK &K,
                                          const double Pg[NV], double P[NV], double &bsq_out,
                                          double &lorentz_out) {
  const double gam = K.gam, igam = K.igam;
#pragma unroll
  for (int v = 0; v < NV; v++) P[v] = Pg[v];
  const double igd = G.igdet;
  const double al = G.alpha;
  P[B1] = U[B1] * igd;
  P[B2] = U[B2] * igd;
  P[B3] = U[B3] * igd;
  const double D = U[RHO] * al * igd;
  if (!(D > 0.0)) return PF_D;
  const double n1 = al * P[B1], n2 = al * P[B2], n3 = al * P[B3];  // normal-frame field
  const double aig = al * igd;
  const double Q1 = aig * U[U1], Q2 = aig * U[U2], Q3 = aig * U[U3];
  // Q'.n = Q.n + D without the rest-mass cancellation
  const double Qpn = (U[UU] - (1.0 - al) * U[RHO]) * igd -
                     al * (Q1 * G.gcon[SY(0, 1)] + Q2 * G.gcon[SY(0, 2)] + Q3 * G.gcon[SY(0, 3)]);
  // spatial inverse metric gamma^{ij} = g^{ij} - g^{it} g^{jt} / g^{tt}, 1/g^{tt} = -alpha^2
  const double ig00 = -al * al;
  const double c1 = G.gcon[SY(0, 1)], c2 = G.gcon[SY(0, 2)], c3 = G.gcon[SY(0, 3)];
  const double h11 = G.gcon[SY(1, 1)] - c1 * c1 * ig00, h12 = G.gcon[SY(1, 2)] - c1 * c2 * ig00;
  const double h13 = G.gcon[SY(1, 3)] - c1 * c3 * ig00, h22 = G.gcon[SY(2, 2)] - c2 * c2 * ig00;
  const double h23 = G.gcon[SY(2, 3)] - c2 * c3 * ig00, h33 = G.gcon[SY(3, 3)] - c3 * c3 * ig00;
  const double Qt1 = h11 * Q1 + h12 * Q2 + h13 * Q3;
  const double Qt2 = h12 * Q1 + h22 * Q2 + h23 * Q3;
  const double Qt3 = h13 * Q1 + h23 * Q2 + h33 * Q3;
  const double Qtsq = Qt1 * Q1 + Qt2 * Q2 + Qt3 * Q3;
  const double QdB = Q1 * n1 + Q2 * n2 + Q3 * n3;
  const double QdB2 = QdB * QdB;
  const double Bsq = n1 * (G.gcov[SY(1, 1)] * n1 + G.gcov[SY(1, 2)] * n2 + G.gcov[SY(1, 3)] * n3) +
                     n2 * (G.gcov[SY(1, 2)] * n1 + G.gcov[SY(2, 2)] * n2 + G.gcov[SY(2, 3)] * n3) +
                     n3 * (G.gcov[SY(1, 3)] * n1 + G.gcov[SY(2, 3)] * n2 + G.gcov[SY(3, 3)] * n3);
  // guess
  const double g1 = Pg[U1], g2 = Pg[U2], g3 = Pg[U3];
  const double qsq = g1 * (G.gcov[SY(1, 1)] * g1 + G.gcov[SY(1, 2)] * g2 + G.gcov[SY(1, 3)] * g3) +
                     g2 * (G.gcov[SY(1, 2)] * g1 + G.gcov[SY(2, 2)] * g2 + G.gcov[SY(2, 3)] * g3) +
                     g3 * (G.gcov[SY(1, 3)] * g1 + G.gcov[SY(2, 3)] * g2 + G.gcov[SY(3, 3)] * g3);
  double Wp = (Pg[RHO] + gam * Pg[UU]) * (1.0 + qsq) - D;
  if (Wp < 0.0) Wp = 0.0;

  const double gf = K.gf;  // (gamma - 1)/gamma
  int converged = 0, extra = 0, invalid = 0, have_hi = 0;
  double lo = 0.0, hi = 0.0;
  for (int it = 0; it < INV_MAXIT + INV_EXTRA; it++) {
    const double W = Wp + D;
    const double W2 = W * W;
    const double BW = Bsq + W;
    const double ix = rcp_nr(BW * W);  // 1/W = BW ix, 1/(B^2+W) = W ix
    const double iBW2W2 = ix * ix;
    double vsq = (Qtsq * W2 + QdB2 * (Bsq + 2.0 * W)) * iBW2W2;
    invalid = 0;
    if (vsq > INV_VSQ_MAX) {
      lo = fmax(lo, Wp);
      Wp = have_hi ? 0.5 * (lo + hi) : Wp + W;
      invalid = 1;
      if (converged || it + 1 >= INV_MAXIT) break;
      continue;
    }
    if (vsq < 0.0) vsq = 0.0;
    const double omv = 1.0 - vsq;
    const double rsq = rsqrt_nr(omv);  // 1/sqrt(1 - v^2)
    const double sq = omv * rsq;
    const double wmr = Wp * omv - D * vsq * sq * rcp_nr(1.0 + sq);
    const double iW = BW * ix;
    const double iW2 = iW * iW;
    const double f = Qpn + Wp - gf * wmr + 0.5 * (1.0 + vsq) * Bsq - 0.5 * QdB2 * iW2;
    if (f > 0.0) {
      hi = have_hi ? fmin(hi, Wp) : Wp;
      have_hi = 1;
    } else {
      lo = fmax(lo, Wp);
    }
    const double dv = -2.0 * (Qtsq * W2 * W + QdB2 * (3.0 * W2 + 3.0 * W * Bsq + Bsq * Bsq)) *
                      (iBW2W2 * ix);
    const double dpdW = gf * (omv + dv * (0.5 * D * rsq - W));
    const double df = 1.0 - dpdW + 0.5 * Bsq * dv + QdB2 * iW2 * iW;
    double Wn = Wp - f * rcp_nr(df);
    if (Wn < 0.0) Wn = 0.5 * Wp;
    if (converged) {
      Wp = Wn;
      if (++extra >= INV_EXTRA) break;
      continue;
    }
    if (fabs(Wn - Wp) <= INV_TOL * fabs(W)) converged = 1;
    Wp = Wn;
    if (!converged && it + 1 >= INV_MAXIT) break;
  }
  const double W = Wp + D;
  if (!converged) return PF_NOCONV;
  if (!(W > 0.0) || !isfinite(W)) return PF_W;
  const double W2 = W * W;
  const double BW = Bsq + W;
  const double ix = rcp_nr(BW * W);
  double vsq = (Qtsq * W2 + QdB2 * (Bsq + 2.0 * W)) * (ix * ix);
  if (!(vsq < 1.0) || invalid) return PF_VSQ;
  if (vsq < 0.0) vsq = 0.0;
  const double omv = 1.0 - vsq;
  const double rsq = rsqrt_nr(omv);  // Lorentz factor
  const double sq = omv * rsq;
  const double rho = D * sq;
  const double uu = (Wp * omv - D * vsq * sq * rcp_nr(1.0 + sq)) * igam;
  if (!(rho > 0.0)) return PF_RHO;
  if (uu < 0.0) return PF_U;
  const double fac = rsq * (W * ix);  // gamma / (W + B^2)
  const double qbw = QdB * (BW * ix);  // Q.B / W
  bsq_out = Bsq * omv + qbw * qbw;
  lorentz_out = rsq;
  P[RHO] = rho;
  P[UU] = uu;
  P[U1] = fac * (Qt1 + qbw * n1);
  P[U2] = fac * (Qt2 + qbw * n2);
  P[U3] = fac * (Qt3 + qbw * n3);
  return PF_OK;
}

// ---------------------------------------------------------------------------
// Bounds: Lorentz-factor cap first (it changes b^2), then rho and u raised in
// the fluid frame in the order of the paper's list; every bound holds on exit.
// ---------------------------------------------------------------------------
// The bounds with b^2 and the Lorentz factor already known (from the
// inversion); zones that need the Lorentz-factor cap take the general path.
// The quotients b^2/sigma, beta b^2 / (2 (gamma - 1)) and u/T are the IEEE
// divisions' values bit for bit (div_rn).
__device__ __forceinline__ int apply_floors(double P[NV], const Geo &G, double rho_fl,
                                            double u_fl, const GasK &K);
__device__ __forceinline__ int apply_floors_known(double P[NV], const Geo &G, double rho_fl,
                                                  double u_fl, const GasK &K, double bsq,
                                                  double lorentz) {
  if (lorentz > FL_GAMMA) return apply_floors(P, G, rho_fl, u_fl, K);
  int fl = 0;
  if (P[RHO] < rho_fl) { P[RHO] = rho_fl; fl |= FF_RHO_GEOM; }
  if (P[UU] < u_fl) { P[UU] = u_fl; fl |= FF_U_GEOM; }
  const double rs = div_rn(bsq, FL_SIGMA, FL_SIGMA_RCP);
  if (P[RHO] < rs) { P[RHO] = rs; fl |= FF_SIGMA; }
  const double ub = div_rn(FL_BETA * bsq, K.ubd, K.ubd_rcp);
  if (P[UU] < ub) { P[UU] = ub; fl |= FF_BETA; }
  const double rt = div_rn(P[UU], FL_TEMP, FL_TEMP_RCP);
  if (P[RHO] < rt) { P[RHO] = rt; fl |= FF_TEMP; }
  return fl;
}

__device__ __forceinline__ int apply_floors(double P[NV], const Geo &G, double rho_fl,
                                            double u_fl, const GasK &K) {
  int fl = 0;
  const double v1 = P[U1], v2 = P[U2], v3 = P[U3];
  const double qsq = v1 * (G.gcov[SY(1, 1)] * v1 + G.gcov[SY(1, 2)] * v2 + G.gcov[SY(1, 3)] * v3) +
                     v2 * (G.gcov[SY(1, 2)] * v1 + G.gcov[SY(2, 2)] * v2 + G.gcov[SY(2, 3)] * v3) +
                     v3 * (G.gcov[SY(1, 3)] * v1 + G.gcov[SY(2, 3)] * v2 + G.gcov[SY(3, 3)] * v3);
  if (sqrt(1.0 + qsq) > FL_GAMMA) {
    const double f = sqrt((FL_GAMMA * FL_GAMMA - 1.0) / qsq);
    P[U1] *= f;
    P[U2] *= f;
    P[U3] *= f;
    fl |= FF_GAMMA;
  }
  FState s;
  fluid_state(P, G, s);
  if (P[RHO] < rho_fl) { P[RHO] = rho_fl; fl |= FF_RHO_GEOM; }
  if (P[UU] < u_fl) { P[UU] = u_fl; fl |= FF_U_GEOM; }
  const double rs = div_rn(s.bsq, FL_SIGMA, FL_SIGMA_RCP);
  if (P[RHO] < rs) { P[RHO] = rs; fl |= FF_SIGMA; }
  const double ub = div_rn(FL_BETA * s.bsq, K.ubd, K.ubd_rcp);
  if (P[UU] < ub) { P[UU] = ub; fl |= FF_BETA; }
  const double rt = div_rn(P[UU], FL_TEMP, FL_TEMP_RCP);
  if (P[RHO] < rt) { P[RHO] = rt; fl |= FF_TEMP; }
  return fl;
}

// Drift-frame bounds.  The mass and internal energy that the fluid-frame
// bounds would add go in as a field-free parcel that moves with the drift
// velocity, the part of the normal-observer 3-velocity v = utilde/gamma
// perpendicular to B; in terms of utilde and the unit field direction Bh,
// utilde_d = (utilde - (utilde.Bh) Bh) / sqrt(1 + (utilde.Bh)^2).  A field
// with g_ij B^i B^j <= 1e-20 rho (rho after the bounds), whose direction
// rounding decides, counts as none: the parcel then moves with the fluid.
// U(P) (after the Lorentz-factor cap) plus
// the parcel's U is inverted from the fluid-frame result, and the fluid-frame
// bounds run once more.  If that inversion fails the fluid-frame result is
// kept.
static __device__ __noinline__ int apply_floors_drift(double P[NV], const Geo &G, double rho_fl,
                                                      double u_fl, const GasK &K) {
  const double gam = K.gam;
  double Pf[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) Pf[v] = P[v];
  int fl = apply_floors(Pf, G, rho_fl, u_fl, K);
  if (!(fl & ~FF_GAMMA)) {
#pragma unroll
    for (int v = 0; v < NV; v++) P[v] = Pf[v];
    return fl;
  }
  double Pc[NV], Pp[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) Pc[v] = P[v];
  Pc[U1] = Pf[U1];
  Pc[U2] = Pf[U2];
  Pc[U3] = Pf[U3];
  Pp[RHO] = Pf[RHO] - Pc[RHO];
  Pp[UU] = Pf[UU] - Pc[UU];
  const double b1 = Pc[B1], b2 = Pc[B2], b3 = Pc[B3];
  const double l1 = G.gcov[SY(1, 1)] * b1 + G.gcov[SY(1, 2)] * b2 + G.gcov[SY(1, 3)] * b3;
  const double l2 = G.gcov[SY(1, 2)] * b1 + G.gcov[SY(2, 2)] * b2 + G.gcov[SY(2, 3)] * b3;
  const double l3 = G.gcov[SY(1, 3)] * b1 + G.gcov[SY(2, 3)] * b2 + G.gcov[SY(3, 3)] * b3;
  const double Bsq = l1 * b1 + l2 * b2 + l3 * b3;
  const double udB = l1 * Pc[U1] + l2 * Pc[U2] + l3 * Pc[U3];
  if (Bsq > FL_DRIFT_BSQ * Pf[RHO]) {
    const double f = 1.0 / sqrt(1.0 + udB * udB / Bsq);
    const double q = udB / Bsq;
    Pp[U1] = f * (Pc[U1] - q * b1);
    Pp[U2] = f * (Pc[U2] - q * b2);
    Pp[U3] = f * (Pc[U3] - q * b3);
  } else {
    Pp[U1] = Pc[U1];
    Pp[U2] = Pc[U2];
    Pp[U3] = Pc[U3];
  }
  Pp[B1] = Pp[B2] = Pp[B3] = 0.0;
  double Us[NV], Up[NV];
  {
    FState s;
    fluid_state(Pc, G, s);
    prim_flux(Pc, s, G, gam, 0, Us);
    fluid_state(Pp, G, s);
    prim_flux(Pp, s, G, gam, 0, Up);
  }
#pragma unroll
  for (int v = 0; v < NV; v++) Us[v] += Up[v];
  double Pn[NV], bsq, lor;
  if (invert_1dw(Us, G, K, Pf, Pn, bsq, lor) != PF_OK) {
#pragma unroll
    for (int v = 0; v < NV; v++) P[v] = Pf[v];
    return fl | FF_DRIFT_FAIL;
  }
  fl |= FF_DRIFT | apply_floors(Pn, G, rho_fl, u_fl, K);
#pragma unroll
  for (int v = 0; v < NV; v++) P[v] = Pn[v];
  return fl;
}

}  // namespace grmhd
