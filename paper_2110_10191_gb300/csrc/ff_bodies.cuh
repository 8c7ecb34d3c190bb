// ff_bodies.cuh -- per-thread bodies of the float-float mode
// (GRMHD_PREC_FF): the reconstruction, the fluid states, the signal speeds,
// the local Lax-Friedrichs flux, U(P), the geometric source and the 1D_W
// inversion in float-float arithmetic (ff.cuh, about 48 significant bits) on
// the FP32 pipe; the state, the fluxes, the flux divergence, the flux-CT and
// the bounds stay FP64.  Same formulas as the FP64 bodies (grmhd_dev.cuh),
// with the energy flux and energy density formed without the rest-mass
// cancellation as in the FP32 bodies (grmhd_f32.cuh), since the 5 bits the
// float pair lacks would otherwise be lost 1e3-fold at rho >> u, and with
// every zone or face computed in units scaled by its density (FFScale).
//
// Data: the stage input split once per stage into high and low float words
// ([2][8][ntot]: all high words, then all low words), the face values in the
// same split layout, and a split copy of the geometry ([2][NLOC][G_NCOMP][n2d]).
#pragma once

#include "ff.cuh"
#include "grmhd_dev.cuh"
#include "step_bodies.cuh"

namespace grmhd {

__device__ __forceinline__ ff ff_load(const float *__restrict__ hi, long long lo_off, long long i) {
  ff r;
  r.hi = __ldg(hi + i);
  r.lo = __ldg(hi + lo_off + i);
  return r;
}

__device__ __forceinline__ void ff_store(float *hi, long long lo_off, long long i, ff v) {
  hi[i] = v.hi;
  hi[lo_off + i] = v.lo;
}

// Per-zone (per-face) scale.  Ideal MHD is invariant under rho, u, p, b^2 ->
// s (rho, u, p, b^2) with B -> sqrt(s) B and the velocities unchanged, so the
// float-float bodies work in units where the density is about 1: s = 4^m
// (an exact power of two whose square root 2^m is exact too) from the
// density; the hydrodynamic densities, fluxes and sources scale by s, the
// field and its fluxes by 2^m.  Without it the float exponent range
// (1e-38..3e38) cuts into floor-density atmospheres, where products such as
// (Q.B)^2 fall below 1e-38.
struct FFScale {
  float is, irs;   // 1/s, 1/sqrt(s): into the scaled units
  double s, rs;    // s, sqrt(s): back, applied in FP64
};

__device__ __forceinline__ FFScale ff_scale_for(float rho) {
  int m = 0;
  if (rho > 0.0f) {
    m = ilogbf(rho) >> 1;  // floor of half the binary exponent
    m = max(-60, min(60, m));
  }
  FFScale c;
  c.is = ldexpf(1.0f, -2 * m);
  c.irs = ldexpf(1.0f, -m);
  c.s = ldexp(1.0, 2 * m);
  c.rs = ldexp(1.0, m);
  return c;
}

// a primitive vector into the scaled units (exact)
__device__ __forceinline__ void ff_scale_prims(ff P[NV], const FFScale &c) {
  P[RHO] = ff_ldexp(P[RHO], c.is);
  P[UU] = ff_ldexp(P[UU], c.is);
  P[B1] = ff_ldexp(P[B1], c.irs);
  P[B2] = ff_ldexp(P[B2], c.irs);
  P[B3] = ff_ldexp(P[B3], c.irs);
}

// one value split into its two words ([2][n]); values beyond the float
// range (inverse-metric components on the polar axis, which no flux reads)
// are clamped to +-FLT_MAX
__device__ __forceinline__ void to_ff_body(const double *__restrict__ src, float *__restrict__ dst,
                                           long long n, long long t) {
  if (t >= n) return;
  const double x = src[t];
  ff v;
  if (fabs(x) > 3.4028234663852886e38) {
    v.hi = (x > 0.0) ? 3.4028234663852886e38f : -3.4028234663852886e38f;
    v.lo = 0.0f;
  } else {
    v = ff_from(x);
  }
  dst[t] = v.hi;
  dst[n + t] = v.lo;
}

// ---------------------------------------------------------------------------
// Reconstruction
// ---------------------------------------------------------------------------
// MC limited slope of x1 with neighbours x0, x2 (the FP64 body's decisions
// taken on the float-float differences)
__device__ __forceinline__ ff mc_slope_ff(ff x0, ff x1, ff x2) {
  const ff dm = ff_sub(x1, x0), dp = ff_sub(x2, x1);
  if (!((dm.hi > 0.0f && dp.hi > 0.0f) || (dm.hi < 0.0f && dp.hi < 0.0f))) return ff_f(0.0f);
  const ff dc = ff_ldexp(ff_add(dm, dp), 0.5f);
  const ff m = ff_min(ff_min(ff_abs(ff_ldexp(dm, 2.0f)), ff_abs(dc)), ff_abs(ff_ldexp(dp, 2.0f)));
  return (dc.hi > 0.0f) ? m : ff_neg(m);
}

// Both WENO5 face values of the middle zone of a..e: the FP64 body's
// first/second-difference form, with the weights d_k/(eps + beta_k)^2
// normalised by the smallest (eps + beta): r_k = min_j e_j / e_k <= 1, so
// no product leaves the float exponent range (eps = 1e-26 makes e_k^2 as
// small as 1e-50); a weight that underflows is negligible next to the
// dominant one, which is 1.
__device__ __forceinline__ void weno5_pair_ff(ff a, ff b, ff c, ff d, ff e, ff &lo, ff &hi) {
  const ff dm2 = ff_sub(b, a), dm1 = ff_sub(c, b), dp1 = ff_sub(d, c), dp2 = ff_sub(e, d);
  const ff D0 = ff_sub(dm1, dm2), D1 = ff_sub(dp1, dm1), D2 = ff_sub(dp2, dp1);
  const ff s0 = ff_add(D0, ff_ldexp(dm1, 2.0f));
  const ff s1 = ff_add(dm1, dp1);
  const ff s2 = ff_sub(D2, ff_ldexp(dp1, 2.0f));
  // 12 (eps + beta_k) = 12 eps + 13 D_k^2 + 3 s_k^2; 12 eps = 1.2e-25 split
  // into its float words (high 0x16148d85, low 0x89c7ce7b: the double
  // constant to 2e-41)
  ff eps12;
  eps12.hi = __int_as_float(0x16148d85);
  eps12.lo = __int_as_float((int)0x89c7ce7bu);
  const ff e0 = ff_add(ff_add(ff_mul_f(ff_sqr(D0), 13.0f), ff_mul_f(ff_sqr(s0), 3.0f)), eps12);
  const ff e1 = ff_add(ff_add(ff_mul_f(ff_sqr(D1), 13.0f), ff_mul_f(ff_sqr(s1), 3.0f)), eps12);
  const ff e2 = ff_add(ff_add(ff_mul_f(ff_sqr(D2), 13.0f), ff_mul_f(ff_sqr(s2), 3.0f)), eps12);
  const ff emin = ff_min(ff_min(e0, e1), e2);
  const ff r0 = ff_mul(emin, ff_rcp(e0)), r1 = ff_mul(emin, ff_rcp(e1)), r2 = ff_mul(emin, ff_rcp(e2));
  const ff w0 = ff_sqr(r0), w1 = ff_mul_f(ff_sqr(r1), 6.0f), w2 = ff_sqr(r2);
  const ff w2x3 = ff_mul_f(w2, 3.0f), w0x3 = ff_mul_f(w0, 3.0f);
  const ff m3 = ff_mul_f(dm1, 3.0f), p3 = ff_mul_f(dp1, 3.0f);
  // high face: linear weights 1 : 6 : 3 on stencils 0, 1, 2
  const ff nh = ff_add(ff_add(ff_mul(w0, ff_add(ff_ldexp(D0, 2.0f), m3)),
                              ff_mul(w1, ff_add(dm1, ff_ldexp(dp1, 2.0f)))),
                       ff_mul(w2x3, ff_sub(p3, D2)));
  const ff H = ff_mul_f(ff_add(ff_add(w0, w1), w2x3), 6.0f);
  // low face: the mirrored stencils (2, 1, 0) with the same linear weights
  const ff nl = ff_sub(ff_sub(ff_mul(w2, ff_sub(ff_ldexp(D2, 2.0f), p3)),
                              ff_mul(w1, ff_add(dp1, ff_ldexp(dm1, 2.0f)))),
                       ff_mul(w0x3, ff_add(m3, D0)));
  const ff L = ff_mul_f(ff_add(ff_add(w2, w1), w0x3), 6.0f);
  hi = ff_add(c, ff_div(nh, H));
  lo = ff_add(c, ff_div(nl, L));
}

// Zone-centric reconstruction along DIR in float-float: Pff is the split
// stage input ([2][8][ntot]), Lf/Rf the split low/high face values.
template <int DIR, int RECON>
__device__ __forceinline__ void recon_ff_body(const StepArgs &A, const float *__restrict__ Pff,
                                              float *__restrict__ Lf, float *__restrict__ Rf,
                                              long long t) {
  const Dims &D = A.D;
  const int e0 = D.n[0] + 2, e1 = D.n[1] + 2;
  if (t >= n_recon(D, A.flat3)) return;
  const int i = NG - 1 + (int)(t % e0);
  const int j = NG - 1 + (int)((t / e0) % e1);
  const int k = (A.flat3 ? NG : NG - 1) + (int)(t / ((long long)e0 * e1));
  const long long c = zid(D, i, j, k);
  const long long st = (DIR == 0) ? 1 : (DIR == 1) ? D.s[0] : D.n2d;
  const long long half = (long long)NV * D.ntot;
#pragma unroll 1
  for (int v = 0; v < NV; v++) {
    const long long o = v * D.ntot + c;
    ff lo, hi;
    if (RECON == 1) {
      weno5_pair_ff(ff_load(Pff, half, o - 2 * st), ff_load(Pff, half, o - st), ff_load(Pff, half, o),
                    ff_load(Pff, half, o + st), ff_load(Pff, half, o + 2 * st), lo, hi);
    } else {
      const ff x1 = ff_load(Pff, half, o);
      const ff h = ff_ldexp(mc_slope_ff(ff_load(Pff, half, o - st), x1, ff_load(Pff, half, o + st)), 0.5f);
      lo = ff_sub(x1, h);
      hi = ff_add(x1, h);
    }
    ff_store(Lf, half, o, lo);
    ff_store(Rf, half, o, hi);
  }
}

// ---------------------------------------------------------------------------
// Face fluxes
// ---------------------------------------------------------------------------
struct GeoFF {
  ff gcov[10], gcon[10], gdet, alpha, ialpha, omalpha, igdet;
};

// geometry of one location from the split copy ([2][NLOC][G_NCOMP][n2d];
// g points at this location's components, lo_off = NLOC G_NCOMP n2d)
__device__ __forceinline__ void load_geo_ff(const float *__restrict__ g, long long lo_off, long long n2d,
                                            long long ij, GeoFF &G) {
#pragma unroll
  for (int q = 0; q < 10; q++) G.gcov[q] = ff_load(g, lo_off, (G_GCOV + q) * n2d + ij);
#pragma unroll
  for (int q = 0; q < 10; q++) G.gcon[q] = ff_load(g, lo_off, (G_GCON + q) * n2d + ij);
  G.gdet = ff_load(g, lo_off, G_GDET * n2d + ij);
  G.alpha = ff_load(g, lo_off, G_ALPHA * n2d + ij);
  G.ialpha = ff_load(g, lo_off, G_IALPHA * n2d + ij);
  G.omalpha = ff_load(g, lo_off, G_OMALPHA * n2d + ij);
  G.igdet = ff_load(g, lo_off, G_IGDET * n2d + ij);
}

// Fluid state as fluid_state (grmhd_dev.cuh), plus opu_t = 1 + u_t formed
// as (1 - alpha) - alpha (gamma - 1) + g_tj utilde^j, gamma - 1 = q^2/(1 + gamma).
struct FStateFF {
  ff ucon[4], ucov[4], bcon[4], bcov[4], bsq, opu_t;
};

__device__ __forceinline__ ff dot3(ff a0, ff b0, ff a1, ff b1, ff a2, ff b2) {
  return ff_add(ff_add(ff_mul(a0, b0), ff_mul(a1, b1)), ff_mul(a2, b2));
}

__device__ __forceinline__ void fluid_state_ff(const ff P[NV], const GeoFF &G, FStateFF &s) {
  const ff v1 = P[U1], v2 = P[U2], v3 = P[U3];
  const ff l1 = dot3(G.gcov[SY(1, 1)], v1, G.gcov[SY(1, 2)], v2, G.gcov[SY(1, 3)], v3);
  const ff l2 = dot3(G.gcov[SY(1, 2)], v1, G.gcov[SY(2, 2)], v2, G.gcov[SY(2, 3)], v3);
  const ff l3 = dot3(G.gcov[SY(1, 3)], v1, G.gcov[SY(2, 3)], v2, G.gcov[SY(3, 3)], v3);
  const ff qsq = dot3(l1, v1, l2, v2, l3, v3);
  const ff g2 = ff_add_f(qsq, 1.0f);
  const ff rg = ff_rsqrt(g2);
  const ff gam = ff_mul(g2, rg);
  const ff ga = ff_mul(gam, G.alpha);
  const ff sh = dot3(G.gcov[SY(0, 1)], v1, G.gcov[SY(0, 2)], v2, G.gcov[SY(0, 3)], v3);
  s.opu_t = ff_add(ff_sub(G.omalpha, ff_mul(ff_mul(G.alpha, qsq), ff_rcp(ff_add_f(gam, 1.0f)))), sh);
  s.ucon[0] = ff_mul(gam, G.ialpha);
  s.ucon[1] = ff_sub(v1, ff_mul(ga, G.gcon[SY(0, 1)]));
  s.ucon[2] = ff_sub(v2, ff_mul(ga, G.gcon[SY(0, 2)]));
  s.ucon[3] = ff_sub(v3, ff_mul(ga, G.gcon[SY(0, 3)]));
  s.ucov[0] = ff_sub(sh, ga);
  s.ucov[1] = l1;
  s.ucov[2] = l2;
  s.ucov[3] = l3;
  const ff bt = dot3(P[B1], l1, P[B2], l2, P[B3], l3);
  const ff iut = ff_mul(G.alpha, rg);  // 1/u^t
  s.bcon[0] = bt;
  s.bcon[1] = ff_mul(ff_add(P[B1], ff_mul(bt, s.ucon[1])), iut);
  s.bcon[2] = ff_mul(ff_add(P[B2], ff_mul(bt, s.ucon[2])), iut);
  s.bcon[3] = ff_mul(ff_add(P[B3], ff_mul(bt, s.ucon[3])), iut);
#pragma unroll
  for (int m = 0; m < 4; m++) {
    ff a = ff_f(0.0f);
#pragma unroll
    for (int n = 0; n < 4; n++) a = ff_add(a, ff_mul(G.gcov[SY(m, n)], s.bcon[n]));
    s.bcov[m] = a;
  }
  s.bsq = ff_add(ff_add(ff_mul(s.bcon[0], s.bcov[0]), ff_mul(s.bcon[1], s.bcov[1])),
                 ff_add(ff_mul(s.bcon[2], s.bcov[2]), ff_mul(s.bcon[3], s.bcov[3])));
}

// acc += F^dir + coef U without the sqrt(-g) factor (flux_cons_acc), the
// energy row as rho uc (1 + u_t) + (w - rho) uc u_t - bc b_t + coef pt
__device__ __forceinline__ void flux_cons_acc_ff(const ff P[NV], const FStateFF &s, ff gm1,
                                                 int dir, ff coef, ff acc[NV]) {
  const ff pg = ff_mul(P[UU], gm1);
  const ff w = ff_add(ff_add(P[RHO], P[UU]), ff_add(pg, s.bsq));
  const ff pt = ff_add(pg, ff_ldexp(s.bsq, 0.5f));
  const ff uc = ff_add(s.ucon[dir], ff_mul(coef, s.ucon[0]));
  const ff bc = ff_add(s.bcon[dir], ff_mul(coef, s.bcon[0]));
  const ff wuc = ff_mul(w, uc);
  ff T[4];
#pragma unroll
  for (int nu = 0; nu < 4; nu++) T[nu] = ff_sub(ff_mul(wuc, s.ucov[nu]), ff_mul(bc, s.bcov[nu]));
  T[dir] = ff_add(T[dir], pt);
  const ff mf = ff_mul(P[RHO], uc);
  acc[RHO] = ff_add(acc[RHO], mf);
  const ff en = ff_add(ff_mul(mf, s.opu_t),
                       ff_sub(ff_mul(ff_mul(ff_sub(w, P[RHO]), uc), s.ucov[0]), ff_mul(bc, s.bcov[0])));
  acc[UU] = ff_add(acc[UU], ff_add(en, ff_mul(coef, pt)));
  acc[U1] = ff_add(acc[U1], T[1]);
  acc[U2] = ff_add(acc[U2], T[2]);
  acc[U3] = ff_add(acc[U3], T[3]);
  acc[B1] = ff_add(acc[B1], ff_sub(ff_mul(s.bcon[1], uc), ff_mul(bc, s.ucon[1])));
  acc[B2] = ff_add(acc[B2], ff_sub(ff_mul(s.bcon[2], uc), ff_mul(bc, s.ucon[2])));
  acc[B3] = ff_add(acc[B3], ff_sub(ff_mul(s.bcon[3], uc), ff_mul(bc, s.ucon[3])));
}

// fast magnetosonic speeds along dir (the quadratic of mhd_cmax)
// gam: the adiabatic index, ggm1 = gam (gam - 1), both float-float
__device__ __forceinline__ void mhd_vchar_ff(const ff P[NV], const FStateFF &s, const GeoFF &G,
                                             ff gam, ff ggm1, int dir, ff &vmax, ff &vmin) {
  // cs2 + va2 - cs2 va2 = (gamma (gamma - 1) u + b^2) / (b^2 + e_f) exactly
  const ff ef = ff_add(P[RHO], ff_mul(P[UU], gam));
  const ff ee = ff_add(s.bsq, ef);
  const ff cms2 = ff_mul(ff_add(ff_mul(P[UU], ggm1), s.bsq), ff_rcp(ee));
  const ff Asq = G.gcon[SY(dir, dir)];
  const ff Bsq = G.gcon[SY(0, 0)];
  const ff AB = G.gcon[SY(0, dir)];
  const ff Au = s.ucon[dir];
  const ff Bu = s.ucon[0];
  const ff AuBu = ff_mul(Au, Bu);
  const ff qa = ff_sub(ff_sqr(Bu), ff_mul(ff_add(Bsq, ff_sqr(Bu)), cms2));
  const ff qb = ff_mul_f(ff_sub(AuBu, ff_mul(ff_add(AB, AuBu), cms2)), -2.0f);
  const ff qc = ff_sub(ff_sqr(Au), ff_mul(ff_add(Asq, ff_sqr(Au)), cms2));
  ff disc = ff_sub(ff_sqr(qb), ff_mul_f(ff_mul(qa, qc), 4.0f));
  disc = (disc.hi > 0.0f) ? ff_sqrt(disc) : ff_f(0.0f);
  const ff i2a = ff_ldexp(ff_rcp(qa), 0.5f);
  const ff v1 = ff_mul(ff_add(ff_neg(qb), disc), i2a);
  const ff v2 = ff_mul(ff_sub(ff_neg(qb), disc), i2a);
  vmax = ff_max(v1, v2);
  vmin = ff_min(v1, v2);
}

// One thread per face: split states Rf(c - st) (left) and Lf(c) (right),
// split geometry; the LLF flux stored in FP64.  Every thread of the block
// must call it (signal-speed block maximum).
template <int DIR>
__device__ __forceinline__ void face_ff_body(const StepArgs &A, const float *__restrict__ geomff,
                                             const float *__restrict__ Lf,
                                             const float *__restrict__ Rf, double *__restrict__ F,
                                             long long t) {
  const Dims &D = A.D;
  int lo[3], ext[3];
  face_box(D, DIR, A.flat3, lo, ext);
  const long long nface = (long long)ext[0] * ext[1] * ext[2];
  const bool active = t < nface;
  double ctop = 0.0;
  if (active) {
    const int i = lo[0] + (int)(t % ext[0]);
    const int j = lo[1] + (int)((t / ext[0]) % ext[1]);
    const int k = lo[2] + (int)(t / ((long long)ext[0] * ext[1]));
    const long long c = zid(D, i, j, k);
    const long long st = (DIR == 0) ? 1 : (DIR == 1) ? D.s[0] : D.n2d;
    const long long half = (long long)NV * D.ntot;
    ff PL[NV], PR[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) {
      PL[v] = ff_load(Rf, half, v * D.ntot + c - st);
      PR[v] = ff_load(Lf, half, v * D.ntot + c);
    }
    const int loc = (DIR == 0) ? LOC_FACE1 : (DIR == 1) ? LOC_FACE2 : LOC_CENT;
    GeoFF G;
    load_geo_ff(geomff + (long long)loc * G_NCOMP * D.n2d, (long long)NLOC * G_NCOMP * D.n2d, D.n2d,
                (long long)j * D.s[0] + i, G);
    const ff gam = {A.gam_ff[0], A.gam_ff[1]}, gm1 = {A.gm1_ff[0], A.gm1_ff[1]};
    const ff ggm1 = {A.ggm1_ff[0], A.ggm1_ff[1]};
    FStateFF sL, sR;
    const FFScale sc = ff_scale_for(PL[RHO].hi);
    ff_scale_prims(PL, sc);
    ff_scale_prims(PR, sc);
    fluid_state_ff(PL, G, sL);
    fluid_state_ff(PR, G, sR);
    ff vmaxL, vminL, vmaxR, vminR;
    mhd_vchar_ff(PL, sL, G, gam, ggm1, DIR + 1, vmaxL, vminL);
    mhd_vchar_ff(PR, sR, G, gam, ggm1, DIR + 1, vmaxR, vminR);
    const ff z = ff_f(0.0f);
    const ff cmax = ff_max(ff_max(z, vmaxL), vmaxR);
    const ff cmin = ff_max(ff_max(z, ff_neg(vminL)), ff_neg(vminR));
    const ff ct = ff_max(cmax, cmin);
    ff acc[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) acc[v] = z;
    flux_cons_acc_ff(PL, sL, gm1, DIR + 1, ct, acc);
    flux_cons_acc_ff(PR, sR, gm1, DIR + 1, ff_neg(ct), acc);
    const ff hg = ff_ldexp(G.gdet, 0.5f);
#pragma unroll
    for (int v = 0; v < NV; v++)
      F[v * D.ntot + c] = ff_to(ff_mul(hg, acc[v])) * (v < B1 ? sc.s : sc.rs);
    if (A.elec_w) {  // the electron entropies' flux weights (rho scales with s)
      const ff wl = ff_mul(hg, ff_mul(PL[RHO], ff_add(sL.ucon[DIR + 1], ff_mul(ct, sL.ucon[0]))));
      const ff wr = ff_mul(hg, ff_mul(PR[RHO], ff_sub(sR.ucon[DIR + 1], ff_mul(ct, sR.ucon[0]))));
      A.elec_w[(2 * DIR) * D.ntot + c] = ff_to(wl) * sc.s;
      A.elec_w[(2 * DIR + 1) * D.ntot + c] = ff_to(wr) * sc.s;
    }
    bool interior = true;
#pragma unroll
    for (int e = 0; e < 3; e++) {
      if (e == DIR) continue;
      const int q = (e == 0) ? i : (e == 1) ? j : k;
      interior = interior && (q >= NG) && (q < D.n[e] + NG);
    }
    if (interior) ctop = ff_to(ct);
  }
  warp_block_max(ctop, &A.clk->ctop_bits[DIR]);
}

// ---------------------------------------------------------------------------
// Update: U(P), the geometric source and the 1D_W inversion in float-float
// ---------------------------------------------------------------------------
// sqrt(-g)-weighted conserved densities of a state (prim_flux with dir 0),
// the energy density without the rest-mass cancellation:
// T^t_t + rho u^t = rho u^t (1 + u_t) + (w - rho) u^t u_t - b^t b_t + p_t
__device__ __forceinline__ void prim_cons_ff(const ff P[NV], const FStateFF &s, const GeoFF &G, ff gm1,
                                             ff U[NV]) {
  const ff pg = ff_mul(P[UU], gm1);
  const ff w = ff_add(ff_add(P[RHO], P[UU]), ff_add(pg, s.bsq));
  const ff pt = ff_add(pg, ff_ldexp(s.bsq, 0.5f));
  const ff ut = s.ucon[0], bt = s.bcon[0];
  const ff wu = ff_mul(w, ut);
  const ff mf = ff_mul(P[RHO], ut);
  U[RHO] = ff_mul(G.gdet, mf);
  const ff en = ff_add(ff_add(ff_mul(mf, s.opu_t), ff_mul(ff_mul(ff_sub(w, P[RHO]), ut), s.ucov[0])),
                       ff_sub(pt, ff_mul(bt, s.bcov[0])));
  U[UU] = ff_mul(G.gdet, en);
#pragma unroll
  for (int i = 1; i < 4; i++) U[UU + i] = ff_mul(G.gdet, ff_sub(ff_mul(wu, s.ucov[i]), ff_mul(bt, s.bcov[i])));
#pragma unroll
  for (int i = 1; i < 4; i++)
    U[B1 + i - 1] = ff_mul(G.gdet, ff_sub(ff_mul(s.bcon[i], ut), ff_mul(bt, s.ucon[i])));
}

// S_nu = sqrt(-g) T^k_l Gamma^l_{nu k} (geo_source) from the split connection
__device__ __forceinline__ void geo_source_ff(const ff P[NV], const FStateFF &s, const GeoFF &G,
                                              const float *__restrict__ connff, long long lo_off,
                                              long long n2d, long long ij, ff gm1, ff S[4]) {
  const ff pg = ff_mul(P[UU], gm1);
  const ff w = ff_add(ff_add(P[RHO], P[UU]), ff_add(pg, s.bsq));
  const ff pt = ff_add(pg, ff_ldexp(s.bsq, 0.5f));
  ff T[4][4];
#pragma unroll
  for (int m = 0; m < 4; m++) {
    const ff wu = ff_mul(w, s.ucon[m]);
#pragma unroll
    for (int n = 0; n < 4; n++) T[m][n] = ff_sub(ff_mul(wu, s.ucov[n]), ff_mul(s.bcon[m], s.bcov[n]));
    T[m][m] = ff_add(T[m][m], pt);
  }
#pragma unroll
  for (int nu = 0; nu < 4; nu++) {
    ff acc = ff_f(0.0f);
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
      for (int l = 0; l < 4; l++)
        acc = ff_add(acc, ff_mul(T[k][l], ff_load(connff, lo_off, (l * 10 + SY(nu, k)) * n2d + ij)));
    S[nu] = ff_mul(acc, G.gdet);
  }
}

// 1D_W inversion (invert_1dw) in float-float: the same iteration rule, the
// same cancellation-free Q'.n and spatial inverse metric; the decisions are
// taken on float-float values against the same constants (split into float
// words: 1 - 1e-10 = 0x3f800000 + 0xaedbe700, 1e-8 = 0x322bcc77 + 0x248c230e).
__device__ __forceinline__ int invert_1dw_ff(const ff U[NV], const GeoFF &G, ff gam, ff igam, ff gf,
                                             const ff Pg[NV], ff P[NV], ff &bsq_out, ff &lorentz_out) {
  const ff vsq_max = {__int_as_float(0x3f800000), __int_as_float((int)0xaedbe700u)};
  const ff tol = {__int_as_float(0x322bcc77), __int_as_float(0x248c230e)};
  const ff z = ff_f(0.0f);
#pragma unroll
  for (int v = 0; v < NV; v++) P[v] = Pg[v];
  const ff igd = G.igdet, al = G.alpha;
  P[B1] = ff_mul(U[B1], igd);
  P[B2] = ff_mul(U[B2], igd);
  P[B3] = ff_mul(U[B3], igd);
  const ff aig = ff_mul(al, igd);
  const ff D = ff_mul(U[RHO], aig);
  if (!(D.hi > 0.0f)) return PF_D;
  const ff n1 = ff_mul(al, P[B1]), n2 = ff_mul(al, P[B2]), n3 = ff_mul(al, P[B3]);
  const ff Q1 = ff_mul(aig, U[U1]), Q2 = ff_mul(aig, U[U2]), Q3 = ff_mul(aig, U[U3]);
  const ff c1 = G.gcon[SY(0, 1)], c2 = G.gcon[SY(0, 2)], c3 = G.gcon[SY(0, 3)];
  const ff Qpn = ff_sub(ff_mul(ff_sub(U[UU], ff_mul(G.omalpha, U[RHO])), igd),
                        ff_mul(al, dot3(Q1, c1, Q2, c2, Q3, c3)));
  const ff mig00 = ff_sqr(al);  // -1/g^tt
  const ff h11 = ff_add(G.gcon[SY(1, 1)], ff_mul(ff_sqr(c1), mig00));
  const ff h12 = ff_add(G.gcon[SY(1, 2)], ff_mul(ff_mul(c1, c2), mig00));
  const ff h13 = ff_add(G.gcon[SY(1, 3)], ff_mul(ff_mul(c1, c3), mig00));
  const ff h22 = ff_add(G.gcon[SY(2, 2)], ff_mul(ff_sqr(c2), mig00));
  const ff h23 = ff_add(G.gcon[SY(2, 3)], ff_mul(ff_mul(c2, c3), mig00));
  const ff h33 = ff_add(G.gcon[SY(3, 3)], ff_mul(ff_sqr(c3), mig00));
  const ff Qt1 = dot3(h11, Q1, h12, Q2, h13, Q3);
  const ff Qt2 = dot3(h12, Q1, h22, Q2, h23, Q3);
  const ff Qt3 = dot3(h13, Q1, h23, Q2, h33, Q3);
  const ff Qtsq = dot3(Qt1, Q1, Qt2, Q2, Qt3, Q3);
  const ff QdB = dot3(Q1, n1, Q2, n2, Q3, n3);
  const ff Bsq = dot3(n1, dot3(G.gcov[SY(1, 1)], n1, G.gcov[SY(1, 2)], n2, G.gcov[SY(1, 3)], n3), n2,
                      dot3(G.gcov[SY(1, 2)], n1, G.gcov[SY(2, 2)], n2, G.gcov[SY(2, 3)], n3), n3,
                      dot3(G.gcov[SY(1, 3)], n1, G.gcov[SY(2, 3)], n2, G.gcov[SY(3, 3)], n3));
  // guess
  const ff g1 = Pg[U1], g2 = Pg[U2], g3 = Pg[U3];
  const ff qsq = dot3(g1, dot3(G.gcov[SY(1, 1)], g1, G.gcov[SY(1, 2)], g2, G.gcov[SY(1, 3)], g3), g2,
                      dot3(G.gcov[SY(1, 2)], g1, G.gcov[SY(2, 2)], g2, G.gcov[SY(2, 3)], g3), g3,
                      dot3(G.gcov[SY(1, 3)], g1, G.gcov[SY(2, 3)], g2, G.gcov[SY(3, 3)], g3));
  ff Wp = ff_sub(ff_mul(ff_add(Pg[RHO], ff_mul(gam, Pg[UU])), ff_add_f(qsq, 1.0f)), D);
  if (Wp.hi < 0.0f) Wp = z;
  int converged = 0, extra = 0, invalid = 0, have_hi = 0;
  ff lo = z, hi = z;
  for (int it = 0; it < INV_MAXIT + INV_EXTRA; it++) {
    const ff W = ff_add(Wp, D);
    const ff W2 = ff_sqr(W);
    const ff BW = ff_add(Bsq, W);
    const ff ix = ff_rcp(ff_mul(BW, W));  // 1/W = BW ix, 1/(B^2+W) = W ix
    const ff a = ff_mul(W, ix);           // 1/(B^2 + W)
    const ff qx = ff_mul(QdB, ix);        // Q.B / (W (B^2 + W))
    // v^2 = Qt^2/(B^2+W)^2 + (Q.B)^2 (B^2 + 2W)/(W^2 (B^2+W)^2), each factor in range
    ff vsq = ff_add(ff_mul(Qtsq, ff_sqr(a)), ff_mul(ff_mul(qx, ff_add(Bsq, ff_ldexp(W, 2.0f))), qx));
    invalid = 0;
    if (ff_gt(vsq, vsq_max)) {
      lo = ff_max(lo, Wp);
      Wp = have_hi ? ff_ldexp(ff_add(lo, hi), 0.5f) : ff_add(Wp, W);
      invalid = 1;
      if (converged || it + 1 >= INV_MAXIT) break;
      continue;
    }
    if (vsq.hi < 0.0f) vsq = z;
    const ff omv = ff_add_f(ff_neg(vsq), 1.0f);
    const ff rsq = ff_rsqrt(omv);  // 1/sqrt(1 - v^2)
    const ff sq = ff_mul(omv, rsq);
    const ff wmr = ff_sub(ff_mul(Wp, omv), ff_mul(ff_mul(ff_mul(D, vsq), sq), ff_rcp(ff_add_f(sq, 1.0f))));
    const ff iW = ff_mul(BW, ix);
    const ff qw0 = ff_mul(QdB, iW);
    const ff f = ff_sub(ff_add(ff_add(Qpn, Wp), ff_mul(ff_ldexp(ff_add_f(vsq, 1.0f), 0.5f), Bsq)),
                        ff_add(ff_mul(gf, wmr), ff_ldexp(ff_sqr(qw0), 0.5f)));
    if (f.hi > 0.0f) {
      hi = have_hi ? ff_min(hi, Wp) : Wp;
      have_hi = 1;
    } else {
      lo = ff_max(lo, Wp);
    }
    const ff poly = ff_add(ff_mul_f(ff_add(W2, ff_mul(W, Bsq)), 3.0f), ff_sqr(Bsq));
    // dv^2/dW = -2 (Qt^2 W^3 + (Q.B)^2 poly) / (W (B^2+W))^3, as
    // -2 [Qt^2 a^3 + qx^2 (poly ix)]
    const ff dv = ff_mul_f(ff_add(ff_mul(ff_mul(Qtsq, a), ff_sqr(a)),
                                  ff_mul(ff_sqr(qx), ff_mul(poly, ix))), -2.0f);
    const ff dpdW = ff_mul(gf, ff_add(omv, ff_mul(dv, ff_sub(ff_mul(ff_ldexp(D, 0.5f), rsq), W))));
    const ff qw = ff_mul(QdB, iW);  // Q.B / W
    const ff df = ff_add(ff_add(ff_add_f(ff_neg(dpdW), 1.0f), ff_mul(ff_ldexp(Bsq, 0.5f), dv)),
                         ff_mul(ff_sqr(qw), iW));
    ff Wn = ff_sub(Wp, ff_div(f, df));
    if (Wn.hi < 0.0f) Wn = ff_ldexp(Wp, 0.5f);
    if (converged) {
      Wp = Wn;
      if (++extra >= INV_EXTRA) break;
      continue;
    }
    if (!ff_gt(ff_abs(ff_sub(Wn, Wp)), ff_mul(tol, ff_abs(W)))) converged = 1;
    Wp = Wn;
    if (!converged && it + 1 >= INV_MAXIT) break;
  }
  const ff W = ff_add(Wp, D);
  if (!converged) return PF_NOCONV;
  if (!(W.hi > 0.0f) || !isfinite(W.hi)) return PF_W;
  const ff BW = ff_add(Bsq, W);
  const ff ix = ff_rcp(ff_mul(BW, W));
  const ff a = ff_mul(W, ix), qx = ff_mul(QdB, ix);
  ff vsq = ff_add(ff_mul(Qtsq, ff_sqr(a)), ff_mul(ff_mul(qx, ff_add(Bsq, ff_ldexp(W, 2.0f))), qx));
  if (!(vsq.hi < 1.0f || (vsq.hi == 1.0f && vsq.lo < 0.0f)) || invalid) return PF_VSQ;
  if (vsq.hi < 0.0f) vsq = z;
  const ff omv = ff_add_f(ff_neg(vsq), 1.0f);
  const ff rsq = ff_rsqrt(omv);  // Lorentz factor
  const ff sq = ff_mul(omv, rsq);
  const ff rho = ff_mul(D, sq);
  const ff uu = ff_mul(ff_sub(ff_mul(Wp, omv), ff_mul(ff_mul(ff_mul(D, vsq), sq), ff_rcp(ff_add_f(sq, 1.0f)))),
                       igam);
  if (!(rho.hi > 0.0f)) return PF_RHO;
  if (uu.hi < 0.0f) return PF_U;
  const ff fac = ff_mul(rsq, ff_mul(W, ix));  // gamma / (W + B^2)
  const ff qbw = ff_mul(QdB, ff_mul(BW, ix));  // Q.B / W
  bsq_out = ff_add(ff_mul(Bsq, omv), ff_sqr(qbw));
  lorentz_out = rsq;
  P[RHO] = rho;
  P[UU] = uu;
  P[U1] = ff_mul(fac, ff_add(Qt1, ff_mul(qbw, n1)));
  P[U2] = ff_mul(fac, ff_add(Qt2, ff_mul(qbw, n2)));
  P[U3] = ff_mul(fac, ff_add(Qt3, ff_mul(qbw, n3)));
  return PF_OK;
}

// One thread per interior zone (update_body): U(P^n) (or its cache), the
// source of P_s, the inversion in float-float; the flux divergence, the
// conserved sum, the bounds and all stored arrays in FP64.  Every thread
// of the block must call it (warp counters).
// Pff (may be null): the split stage input of the flux stage, which is P_s:
// the update reads P_s's words there instead of splitting P_s again (in the
// predictor P_s = P_i = P^n).  Ucache holds U(P^n) as split words in P^n's scaled
// units ([2][8][ntot] floats in the space of [8][ntot] doubles): the
// corrector, which scales by the same P^n density, reads it back as is.
__device__ __forceinline__ void update_ff_body(const StepArgs &A, const double *Pi,
                                               const double *__restrict__ Ps, double *Pout,
                                               const double *__restrict__ F1,
                                               const double *__restrict__ F2,
                                               const double *__restrict__ F3, int *pflag, int *fflag,
                                               double dtfac, double *Ucache, int ucache_mode,
                                               const float *__restrict__ Pff, long long t) {
  const Dims &D = A.D;
  const double dt = A.clk->dt;
  if (!(dt > 0.0)) return;  // uniform across the grid
  const double dtp = dtfac * dt;
  const long long nz = n_zone(D);
  const bool active = t < nz;
  int pf = 0, fl = 0;
  if (active) {
    const int i = NG + (int)(t % D.n[0]);
    const int j = NG + (int)((t / D.n[0]) % D.n[1]);
    const int k = NG + (int)(t / ((long long)D.n[0] * D.n[1]));
    const long long c = zid(D, i, j, k), N = D.ntot;
    const long long ij = (long long)j * D.s[0] + i;
    GeoFF G;
    load_geo_ff(A.geomff, (long long)NLOC * G_NCOMP * D.n2d, D.n2d, ij, G);
    const ff gam = {A.gam_ff[0], A.gam_ff[1]}, gm1 = {A.gm1_ff[0], A.gm1_ff[1]};
    const ff igam = {A.igam_ff[0], A.igam_ff[1]}, gf = {A.gf_ff[0], A.gf_ff[1]};
    const long long clo = (long long)C_NCOMP * D.n2d;
    ff pi[NV], Ui[NV], S[4];
    if (Ps == Pi && Pff) {
#pragma unroll
      for (int v = 0; v < NV; v++) pi[v] = ff_load(Pff, (long long)NV * N, v * N + c);
    } else {
#pragma unroll
      for (int v = 0; v < NV; v++) pi[v] = ff_from(Pi[v * N + c]);
    }
    float *Ucf = reinterpret_cast<float *>(Ucache);
    const long long uhalf = (long long)NV * N;
    // scaled units from P^n's density (the same in both stages, so that
    // U(P^n) kept by the predictor is read back in the corrector's units)
    const FFScale sc = ff_scale_for(pi[RHO].hi);
    ff_scale_prims(pi, sc);
    if (Ps == Pi) {
      FStateFF si;
      fluid_state_ff(pi, G, si);
      prim_cons_ff(pi, si, G, gm1, Ui);
      if (ucache_mode == 1) {
#pragma unroll
        for (int v = 0; v < NV; v++) ff_store(Ucf, uhalf, v * N + c, Ui[v]);
      }
      geo_source_ff(pi, si, G, A.connff, clo, D.n2d, ij, gm1, S);
    } else {
      if (ucache_mode == 2) {
#pragma unroll
        for (int v = 0; v < NV; v++) Ui[v] = ff_load(Ucf, uhalf, v * N + c);
      } else {
        FStateFF si;
        fluid_state_ff(pi, G, si);
        prim_cons_ff(pi, si, G, gm1, Ui);
      }
      ff ps[NV];
      if (Pff) {  // the corrector's flux stage split P_s
#pragma unroll
        for (int v = 0; v < NV; v++) ps[v] = ff_load(Pff, (long long)NV * N, v * N + c);
      } else {
#pragma unroll
        for (int v = 0; v < NV; v++) ps[v] = ff_from(Ps[v * N + c]);
      }
      ff_scale_prims(ps, sc);
      FStateFF ss;
      fluid_state_ff(ps, G, ss);
      geo_source_ff(ps, ss, G, A.connff, clo, D.n2d, ij, gm1, S);
    }
    const double idx1 = A.idx[0], idx2 = A.idx[1], idx3 = A.idx[2];
    const ff dtpf = ff_from(dtp);
    // The field is updated in FP64, sqrt(-g) B (P^n) - dt' div F_B, as the
    // FP64 update does: flux-CT's divergence-free increments then keep div B
    // at FP64 round-off; the inversion reads the result's words.
    const double gdd = __ldg(A.geom + (long long)G_GDET * D.n2d + ij);
    const double igdd = __ldg(A.geom + (long long)G_IGDET * D.n2d + ij);
    double UB[3];
    ff Un[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) {
      const long long o = v * N + c;
      const double div = (F1[o + 1] - F1[o]) * idx1 + (F2[o + D.s[0]] - F2[o]) * idx2 +
                         (F3[o + D.n2d] - F3[o]) * idx3;
      if (v >= B1) {
        UB[v - B1] = gdd * Pi[o] + dtp * (0.0 - div);
        Un[v] = ff_from(UB[v - B1] * (double)sc.irs);
        continue;
      }
      ff rhs = ff_neg(ff_from(div * (double)sc.is));
      if (v >= UU && v <= U3) rhs = ff_add(rhs, S[v - UU]);
      Un[v] = ff_add(Ui[v], ff_mul(dtpf, rhs));
    }
    ff pn[NV], bsq_n = ff_f(0.0f), lor_n = ff_f(1.0f);
    pf = invert_1dw_ff(Un, G, gam, igam, gf, pi, pn, bsq_n, lor_n);
    double pd[NV];
#pragma unroll
    for (int v = 0; v < B1; v++) {
      pd[v] = ff_to(pn[v]);
      if (v == RHO || v == UU) pd[v] *= sc.s;
    }
#pragma unroll
    for (int q = 0; q < 3; q++) pd[B1 + q] = UB[q] * igdd;
    if (pf == PF_OK && A.floors_on && !A.floor_drift && !A.elec) {
      const double rho_fl = __ldg(A.floors + ij), u_fl = __ldg(A.floors + D.n2d + ij);
      const double lor = ff_to(lor_n);
      if (lor > FL_GAMMA) {  // the Lorentz-factor cap needs the FP64 fluid state
        Geo Gd;
        load_geo(A.geom, D.n2d, ij, Gd);
        fl = apply_floors(pd, Gd, rho_fl, u_fl, A.gk);
      } else {
        Geo Gd;  // not read on this path
        fl = apply_floors_known(pd, Gd, rho_fl, u_fl, A.gk, ff_to(bsq_n) * sc.s, lor);
      }
    }
#pragma unroll
    for (int v = 0; v < NV; v++) Pout[v * N + c] = pd[v];
    pflag[c] = pf;
    fflag[c] = fl;
  }
  count_warp(active && pf != 0, &A.clk->counters[0]);
  count_warp(active && fl != 0, &A.clk->counters[1]);
}

}  // namespace grmhd
