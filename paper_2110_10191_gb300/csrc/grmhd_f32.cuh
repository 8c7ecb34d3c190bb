// grmhd_f32.cuh -- FP32 versions of the face-flux physics for the mixed
// precision mode: reconstruction, fluid state, signal speeds and the local
// Lax-Friedrichs flux run on the FP32 pipe (64x the FP64 rate on GB300);
// the geometry, flux-CT EMFs, conserved update, 1D_W inversion and bounds
// stay FP64.  Same formulas as grmhd_dev.cuh.
#pragma once

#include <cfloat>

#include "grmhd_dev.cuh"

namespace grmhd {

// FP32 reciprocal: the hardware approximation (PTX rcp.approx.ftz.f32,
// within one ulp of 1/x), one instruction against the IEEE sequence of
// __frcp_rn; the FP32 flux stage rounds at that level anyway.  Every
// caller passes a normal, non-zero argument (the WENO variation is at least
// 1e-30, the smoothness indicators at least their epsilon, the signal-speed
// denominators are sums of positive terms).
__device__ __forceinline__ float rcp_f(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

struct GeoF {
  float gcov[10], gcon[10], gdet, alpha, ialpha, omalpha;
};

// geometry in float: [NLOC][G_NCOMP][n2d] like the FP64 copy
__device__ __forceinline__ void load_geo_f(const float *__restrict__ g, long long n2d, long long ij,
                                           GeoF &G) {
#pragma unroll
  for (int c = 0; c < 10; c++) G.gcov[c] = __ldg(g + (G_GCOV + c) * n2d + ij);
#pragma unroll
  for (int c = 0; c < 10; c++) G.gcon[c] = __ldg(g + (G_GCON + c) * n2d + ij);
  G.gdet = __ldg(g + G_GDET * n2d + ij);
  G.alpha = __ldg(g + G_ALPHA * n2d + ij);
  G.ialpha = __ldg(g + G_IALPHA * n2d + ij);
  G.omalpha = __ldg(g + G_OMALPHA * n2d + ij);
}

// opu_t = 1 + u_t, formed without the cancellation of the rest mass:
// (1 - alpha) - alpha (gamma - 1) + g_tj utilde^j with gamma - 1 = q^2/(1 + gamma).
struct FStateF {
  float ucon[4], ucov[4], bcon[4], bcov[4], bsq, opu_t;
};

__device__ __forceinline__ void fluid_state_f(const float P[NV], const GeoF &G, FStateF &s) {
  const float v1 = P[U1], v2 = P[U2], v3 = P[U3];
  const float l1 = G.gcov[SY(1, 1)] * v1 + G.gcov[SY(1, 2)] * v2 + G.gcov[SY(1, 3)] * v3;
  const float l2 = G.gcov[SY(1, 2)] * v1 + G.gcov[SY(2, 2)] * v2 + G.gcov[SY(2, 3)] * v3;
  const float l3 = G.gcov[SY(1, 3)] * v1 + G.gcov[SY(2, 3)] * v2 + G.gcov[SY(3, 3)] * v3;
  const float qsq = l1 * v1 + l2 * v2 + l3 * v3;
  const float g2 = 1.0f + qsq;
  const float rg = rsqrtf(g2);
  const float gam = g2 * rg;
  const float ga = gam * G.alpha;
  const float sh = G.gcov[SY(0, 1)] * v1 + G.gcov[SY(0, 2)] * v2 + G.gcov[SY(0, 3)] * v3;
  s.opu_t = G.omalpha - G.alpha * qsq * rcp_f(1.0f + gam) + sh;
  s.ucon[0] = gam * G.ialpha;
  s.ucon[1] = v1 - ga * G.gcon[SY(0, 1)];
  s.ucon[2] = v2 - ga * G.gcon[SY(0, 2)];
  s.ucon[3] = v3 - ga * G.gcon[SY(0, 3)];
  s.ucov[0] = -ga + sh;
  s.ucov[1] = l1;
  s.ucov[2] = l2;
  s.ucov[3] = l3;
  const float bt = P[B1] * l1 + P[B2] * l2 + P[B3] * l3;
  const float iut = G.alpha * rg;
  s.bcon[0] = bt;
  s.bcon[1] = (P[B1] + bt * s.ucon[1]) * iut;
  s.bcon[2] = (P[B2] + bt * s.ucon[2]) * iut;
  s.bcon[3] = (P[B3] + bt * s.ucon[3]) * iut;
#pragma unroll
  for (int m = 0; m < 4; m++) {
    float a = 0.0f;
#pragma unroll
    for (int n = 0; n < 4; n++) a += G.gcov[SY(m, n)] * s.bcon[n];
    s.bcov[m] = a;
  }
  s.bsq = s.bcon[0] * s.bcov[0] + s.bcon[1] * s.bcov[1] + s.bcon[2] * s.bcov[2] +
          s.bcon[3] * s.bcov[3];
}

__device__ __forceinline__ void flux_cons_acc_f(const float P[NV], const FStateF &s, float gam,
                                                int dir, float coef, float acc[NV]) {
  const float pg = (gam - 1.0f) * P[UU];
  const float w = P[RHO] + P[UU] + pg + s.bsq;
  const float pt = pg + 0.5f * s.bsq;
  const float uc = s.ucon[dir] + coef * s.ucon[0];
  const float bc = s.bcon[dir] + coef * s.bcon[0];
  const float wuc = w * uc;
  float T[4];
#pragma unroll
  for (int nu = 0; nu < 4; nu++) T[nu] = wuc * s.ucov[nu] - bc * s.bcov[nu];
  T[dir] += pt;
  T[0] += coef * pt;
  const float mf = P[RHO] * uc;
  acc[RHO] += mf;
  // T^d_t + rho u^d = rho uc (1 + u_t) + (w - rho) uc u_t - bc b_t (+ pressure term)
  acc[UU] += mf * s.opu_t + ((w - P[RHO]) * uc * s.ucov[0] - bc * s.bcov[0]) + coef * pt;
  acc[U1] += T[1];
  acc[U2] += T[2];
  acc[U3] += T[3];
  acc[B1] += s.bcon[1] * uc - bc * s.ucon[1];
  acc[B2] += s.bcon[2] * uc - bc * s.ucon[2];
  acc[B3] += s.bcon[3] * uc - bc * s.ucon[3];
}

__device__ __forceinline__ void mhd_vchar_f(const float P[NV], const FStateF &s, const GeoF &G,
                                            float gam, int dir, float &vmax, float &vmin) {
  const float ef = P[RHO] + gam * P[UU];
  const float ee = s.bsq + ef;
  const float iee = rcp_f(fmaxf(ef * ee, FLT_MIN));  // (densities below ~1e-19 stay normal)
  const float va2 = s.bsq * ef * iee;
  const float cs2 = gam * (gam - 1.0f) * P[UU] * ee * iee;
  const float cms2 = cs2 + va2 - cs2 * va2;
  const float Asq = G.gcon[SY(dir, dir)];
  const float Bsq = G.gcon[SY(0, 0)];
  const float AB = G.gcon[SY(0, dir)];
  const float Au = s.ucon[dir];
  const float Bu = s.ucon[0];
  const float AuBu = Au * Bu;
  const float qa = Bu * Bu - (Bsq + Bu * Bu) * cms2;
  const float qb = -2.0f * (AuBu - (AB + AuBu) * cms2);
  const float qc = Au * Au - (Asq + Au * Au) * cms2;
  float disc = qb * qb - 4.0f * qa * qc;
  disc = (disc > 0.0f) ? sqrtf(disc) : 0.0f;
  const float i2a = 0.5f * rcp_f(qa);
  const float v1 = (-qb + disc) * i2a;
  const float v2 = (-qb - disc) * i2a;
  vmax = fmaxf(v1, v2);
  vmin = fminf(v1, v2);
}

__device__ __forceinline__ float mc_slope_f(float x0, float x1, float x2) {
  const float dm = x1 - x0, dp = x2 - x1;
  if (!(dm * dp > 0.0f)) return 0.0f;
  const float dc = 0.5f * (dm + dp);
  const float m = fminf(fminf(fabsf(2.0f * dm), fabsf(dc)), fabsf(2.0f * dp));
  return (dc > 0.0f) ? m : -m;
}

// Both WENO5 face values in FP32.  The first and second differences are
// scaled by the local variation s so that the smoothness indicators stay in
// range; the FP64 epsilon (1e-26, absolute) becomes 12e-26/s^2 in these
// units, kept within [1e-30, 1e8] (at 1e8 the weights equal the linear
// weights to FP32 precision).  The weights d_k/e_k^2 are normalised by the
// smallest e_k, so the dominant stencil has weight d_k and the others
// cannot overflow.  Constant data (s <= 1e-30) returns c.
__device__ __forceinline__ void weno5_pair_f(float a, float b, float c, float d, float e, float &lo,
                                             float &hi) {
  float dm2 = b - a, dm1 = c - b, dp1 = d - c, dp2 = e - d;
  const float sc = fmaxf(fmaxf(fabsf(dm2), fabsf(dm1)), fmaxf(fabsf(dp1), fabsf(dp2)));
  // a variation below 1e-30 (e.g. a field tail stored as an FP32 subnormal,
  // whose reciprocal would overflow) is constant data at FP32 precision
  if (!(sc > 1.0e-30f)) {
    lo = c;
    hi = c;
    return;
  }
  const float is = rcp_f(sc);
  dm2 *= is;
  dm1 *= is;
  dp1 *= is;
  dp2 *= is;
  const float eps = fmaxf(fminf(12.0e-26f * is * is, 1.0e8f), 1.0e-30f);
  const float D0 = dm1 - dm2, D1 = dp1 - dm1, D2 = dp2 - dp1;
  const float s0 = D0 + 2.0f * dm1, s1 = dm1 + dp1, s2 = D2 - 2.0f * dp1;
  const float e0 = eps + (13.0f * D0 * D0 + 3.0f * s0 * s0);
  const float e1 = eps + (13.0f * D1 * D1 + 3.0f * s1 * s1);
  const float e2 = eps + (13.0f * D2 * D2 + 3.0f * s2 * s2);
  const float emin = fminf(fminf(e0, e1), e2);
  const float r0 = emin * rcp_f(e0), r1 = emin * rcp_f(e1), r2 = emin * rcp_f(e2);
  const float w0 = r0 * r0, w1 = 6.0f * (r1 * r1), w2 = r2 * r2;
  const float m3 = 3.0f * dm1, p3 = 3.0f * dp1;
  // high face: linear weights 1 : 6 : 3 on stencils 0, 1, 2
  const float nh = w0 * (2.0f * D0 + m3) + w1 * (dm1 + 2.0f * dp1) + 3.0f * w2 * (p3 - D2);
  const float H = 6.0f * (w0 + w1 + 3.0f * w2);
  // low face: the mirrored stencils (2, 1, 0) with the same linear weights
  const float nl = w2 * (2.0f * D2 - p3) - w1 * (dp1 + 2.0f * dm1) - 3.0f * w0 * (m3 + D0);
  const float L = 6.0f * (w2 + w1 + 3.0f * w0);
  hi = c + sc * (nh * rcp_f(H));
  lo = c + sc * (nl * rcp_f(L));
}

}  // namespace grmhd
