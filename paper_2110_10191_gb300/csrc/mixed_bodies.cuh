// mixed_bodies.cuh -- per-thread bodies of the flux stage of the mixed
// precision mode.
//
// An FP32 copy of the primitives (with ghosts) and of the geometry feeds a
// zone-centric FP32 reconstruction and an FP32 face-flux body (fluid state,
// signal speeds, local Lax-Friedrichs flux); the fluxes are written in FP64,
// so the flux-CT EMF combination, the conserved-variable accumulation, the
// 1D_W inversion and the bounds run in FP64 as in the full-FP64 mode.  The
// signal-speed maxima for the time step come from the FP32 states.  Index
// ranges (and the flat-X3 mode) are those of step_bodies.cuh.
#pragma once

#include <cfloat>

#include "grmhd_f32.cuh"
#include "step_bodies.cuh"

namespace grmhd {

// FP64 -> FP32, clamped to the float range (metric components at the poles)
__device__ __forceinline__ void to_f32_body(const double *__restrict__ src, float *__restrict__ dst,
                                            long long n, long long t) {
  if (t >= n) return;
  const double x = src[t];
  dst[t] = (float)fmax(fmin(x, (double)FLT_MAX), -(double)FLT_MAX);
}

template <int DIR, int RECON>
__device__ __forceinline__ void recon_f32_body(const StepArgs &A, const float *__restrict__ P,
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
#pragma unroll
  for (int v = 0; v < NV; v++) {
    const float *p = P + v * D.ntot + c;
    float lo, hi;
    if (RECON == 1) {
      weno5_pair_f(__ldg(p - 2 * st), __ldg(p - st), __ldg(p), __ldg(p + st), __ldg(p + 2 * st), lo,
                   hi);
    } else {
      const float x1 = __ldg(p), h = 0.5f * mc_slope_f(__ldg(p - st), x1, __ldg(p + st));
      lo = x1 - h;
      hi = x1 + h;
    }
    Lf[v * D.ntot + c] = lo;
    Rf[v * D.ntot + c] = hi;
  }
}

// Every thread of the block must call it (signal-speed block maximum).
template <int DIR>
__device__ __forceinline__ void face_f32_body(const StepArgs &A, const float *__restrict__ geomf,
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
    float PL[NV], PR[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) {
      PL[v] = __ldg(Rf + v * D.ntot + c - st);
      PR[v] = __ldg(Lf + v * D.ntot + c);
    }
    const int loc = (DIR == 0) ? LOC_FACE1 : (DIR == 1) ? LOC_FACE2 : LOC_CENT;
    GeoF G;
    load_geo_f(geomf + (long long)loc * G_NCOMP * D.n2d, D.n2d, (long long)j * D.s[0] + i, G);
    const float gam = (float)A.gam;
    FStateF sL, sR;
    fluid_state_f(PL, G, sL);
    fluid_state_f(PR, G, sR);
    float vmaxL, vminL, vmaxR, vminR;
    mhd_vchar_f(PL, sL, G, gam, DIR + 1, vmaxL, vminL);
    mhd_vchar_f(PR, sR, G, gam, DIR + 1, vmaxR, vminR);
    const float cmax = fmaxf(fmaxf(0.0f, vmaxL), vmaxR);
    const float cmin = fmaxf(fmaxf(0.0f, -vminL), -vminR);
    const float ct = fmaxf(cmax, cmin);
    float acc[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) acc[v] = 0.0f;
    flux_cons_acc_f(PL, sL, gam, DIR + 1, ct, acc);
    flux_cons_acc_f(PR, sR, gam, DIR + 1, -ct, acc);
    const float hg = 0.5f * G.gdet;
#pragma unroll
    for (int v = 0; v < NV; v++) F[v * D.ntot + c] = (double)(hg * acc[v]);
    if (A.elec_w) {  // the electron entropies' flux weights, in FP32 as the fluxes
      A.elec_w[(2 * DIR) * D.ntot + c] = (double)(hg * (PL[RHO] * (sL.ucon[DIR + 1] + ct * sL.ucon[0])));
      A.elec_w[(2 * DIR + 1) * D.ntot + c] =
          (double)(hg * (PR[RHO] * (sR.ucon[DIR + 1] - ct * sR.ucon[0])));
    }
    bool interior = true;
#pragma unroll
    for (int e = 0; e < 3; e++) {
      if (e == DIR) continue;
      const int q = (e == 0) ? i : (e == 1) ? j : k;
      interior = interior && (q >= NG) && (q < D.n[e] + NG);
    }
    if (interior) ctop = (double)ct;
  }
  warp_block_max(ctop, &A.clk->ctop_bits[DIR]);
}

}  // namespace grmhd
