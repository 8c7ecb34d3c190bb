// mixed_bodies.cuh -- per-thread bodies of the flux stage of the mixed
// precision mode.
//
// An FP32 copy of the primitives (with ghosts) and of the geometry feeds a
// fused FP32 kernel per direction: each thread reconstructs zones (MC or
// WENO5, both face values of a zone from one stencil) and combines the high
// face value of one zone with the low face value of the next into the fluid
// states, signal speeds and local Lax-Friedrichs flux of the face between
// them.  The face values never leave the SM: the zone-centric face values
// of the FP64 path go through HBM (8 x 2 values per zone written, then read
// by the face kernel), which in FP32 costs more than the arithmetic.
//
//   X1: one thread per zone of the reconstruction range, flattened with i
//       fastest, in warps of 32 consecutive zones that overlap by one: lane
//       l takes the high face value of lane l-1 by a warp shuffle, and lane
//       0 only reconstructs (its zone is the last of the previous warp).
//   X2, X3: one thread per column of faces (i fastest across the threads of
//       a warp, so loads coalesce) and segment of WALK faces along the
//       direction; the thread walks the segment, keeping the high face value
//       of the zone below in registers, after reconstructing one zone below
//       the segment.
//
// The fluxes are written in FP64, so the flux-CT EMF combination, the
// conserved-variable accumulation, the 1D_W inversion and the bounds run in
// FP64 as in the full-FP64 mode.  The signal-speed maxima for the time step
// come from the FP32 states.  Face ranges (and the flat-X3 mode) are those of
// step_bodies.cuh: with flat X3 the X3 faces of the single layer take the
// reconstruction of data that is constant along X3, which returns the data
// exactly (as the FP64 path's direct reads of the primitives).
#pragma once

#include <cfloat>

#include "grmhd_f32.cuh"
#include "step_bodies.cuh"

namespace grmhd {

constexpr int WALK = 16;  // faces per thread along X2 and X3

// FP64 -> FP32, clamped to the float range (metric components at the poles)
__device__ __forceinline__ void to_f32_body(const double *__restrict__ src, float *__restrict__ dst,
                                            long long n, long long t) {
  if (t >= n) return;
  const double x = src[t];
  dst[t] = (float)fmax(fmin(x, (double)FLT_MAX), -(double)FLT_MAX);
}

// FP64 -> FP32 copy of a stage input (primitives: all inside the float
// range), two elements per thread (n even; 16-byte aligned arrays), one
// conversion each: on GB300 the conversion runs on the FP64 pipe, and the
// clamp of to_f32_body would triple its work.
__device__ __forceinline__ void to_f32_state_body(const double *__restrict__ src,
                                                  float *__restrict__ dst, long long n,
                                                  long long t) {
  if (2 * t >= n) return;
  const double2 x = reinterpret_cast<const double2 *>(src)[t];
  reinterpret_cast<float2 *>(dst)[t] = make_float2((float)x.x, (float)x.y);
}

// Both face values (lo: low face, hi: high face) of the 8 primitives of
// zone c along DIR (stride st).
template <int RECON>
__device__ __forceinline__ void recon_zone_f32(const Dims &D, const float *__restrict__ P,
                                               long long c, long long st, float lo[NV],
                                               float hi[NV]) {
#pragma unroll
  for (int v = 0; v < NV; v++) {
    const float *p = P + v * D.ntot + c;
    if (RECON == 1) {
      weno5_pair_f(__ldg(p - 2 * st), __ldg(p - st), __ldg(p), __ldg(p + st), __ldg(p + 2 * st),
                   lo[v], hi[v]);
    } else {
      const float x1 = __ldg(p), h = 0.5f * mc_slope_f(__ldg(p - st), x1, __ldg(p + st));
      lo[v] = x1 - h;
      hi[v] = x1 + h;
    }
  }
}

// The LLF flux of the face at zone c (index (i, j, k)) along DIR between the
// states PL (below) and PR (above), stored in FP64; returns the face's
// signal speed if its transverse indices are interior (it enters the time
// step), else 0.
template <int DIR>
__device__ __forceinline__ double face_flux_f32(const StepArgs &A, const float *__restrict__ geomf,
                                                const float PL[NV], const float PR[NV],
                                                double *__restrict__ F, int i, int j, int k,
                                                long long c) {
  const Dims &D = A.D;
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
  return interior ? (double)ct : 0.0;
}

// Threads of the fused X1 kernel: warps of 32 lanes over 31 new zones each
// of the reconstruction range (the face range with one more zone below it
// along X1).
__host__ __device__ inline long long n_flux_f32_x1(const Dims &D, int flat3) {
  int lo[3], ext[3];
  face_box(D, 0, flat3, lo, ext);
  const long long z = (long long)(ext[0] + 1) * ext[1] * ext[2];
  return 32 * ((z + 30) / 31);
}

// Threads of the fused X2 / X3 kernels: one per column of faces and segment
// of WALK faces along the direction.
__host__ __device__ inline long long n_flux_f32_walk(const Dims &D, int dir, int flat3) {
  int lo[3], ext[3];
  face_box(D, dir, flat3, lo, ext);
  const int b = (dir == 1) ? 2 : 1;
  return (long long)ext[0] * ext[b] * ((ext[dir] + WALK - 1) / WALK);
}

// Fused X1 reconstruction and face fluxes.  Every thread of the block must
// call it (warp shuffle, signal-speed block maximum); the block size is a
// multiple of 32, so t & 31 is the hardware lane.
template <int RECON>
__device__ __forceinline__ void flux_f32_x1_body(const StepArgs &A, const float *__restrict__ geomf,
                                                 const float *__restrict__ P,
                                                 double *__restrict__ F, long long t) {
  const Dims &D = A.D;
  int lo[3], ext[3];
  face_box(D, 0, A.flat3, lo, ext);
  const int e0 = ext[0] + 1;  // zones lo[0]-1 .. lo[0]+ext[0]-1 along X1
  const long long z = (long long)e0 * ext[1] * ext[2];
  const int lane = (int)(t & 31);
  const long long q = 31 * (t >> 5) - 1 + lane;
  const bool have = q >= 0 && q < z;
  float zl[NV], zh[NV];
  int i = 0, j = 0, k = 0, ii = 0;
  long long c = 0;
  if (have) {
    ii = (int)(q % e0);
    i = lo[0] - 1 + ii;
    j = lo[1] + (int)((q / e0) % ext[1]);
    k = lo[2] + (int)(q / ((long long)e0 * ext[1]));
    c = zid(D, i, j, k);
    recon_zone_f32<RECON>(D, P, c, 1, zl, zh);
  } else {
#pragma unroll
    for (int v = 0; v < NV; v++) zl[v] = zh[v] = 0.0f;
  }
  // the high face value of the zone below (lane - 1; same row when ii > 0)
  float PL[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) PL[v] = __shfl_up_sync(0xffffffffu, zh[v], 1);
  double ctop = 0.0;
  if (have && lane > 0 && ii > 0) ctop = face_flux_f32<0>(A, geomf, PL, zl, F, i, j, k, c);
  warp_block_max(ctop, &A.clk->ctop_bits[0]);
}

// Fused X2 / X3 reconstruction and face fluxes, one column segment per
// thread.  Every thread of the block must call it (signal-speed block
// maximum).
template <int DIR, int RECON>
__device__ __forceinline__ void flux_f32_walk_body(const StepArgs &A,
                                                   const float *__restrict__ geomf,
                                                   const float *__restrict__ P,
                                                   double *__restrict__ F, long long t) {
  const Dims &D = A.D;
  int lo[3], ext[3];
  face_box(D, DIR, A.flat3, lo, ext);
  const int b = (DIR == 1) ? 2 : 1;  // the transverse axis beside X1
  const long long ncol = (long long)ext[0] * ext[b];
  const int nseg = (ext[DIR] + WALK - 1) / WALK;
  double ctop = 0.0;
  if (t < ncol * nseg) {
    const long long col = t % ncol;
    const int seg = (int)(t / ncol);
    const int i = lo[0] + (int)(col % ext[0]);
    const int tb = lo[b] + (int)(col / ext[0]);
    const int f0 = seg * WALK, f1 = min(f0 + WALK, ext[DIR]);
    const long long st = (DIR == 1) ? D.s[0] : D.n2d;
    const int j0 = (DIR == 1) ? lo[1] + f0 : tb, k0 = (DIR == 1) ? tb : lo[2] + f0;
    long long c = zid(D, i, j0, k0) - st;  // the zone below the segment's first face
    float zl[NV], zh[NV], PL[NV];
    recon_zone_f32<RECON>(D, P, c, st, zl, PL);
    for (int f = f0; f < f1; f++) {
      c += st;
      recon_zone_f32<RECON>(D, P, c, st, zl, zh);
      const int jf = (DIR == 1) ? lo[1] + f : tb, kf = (DIR == 1) ? tb : lo[2] + f;
      ctop = fmax(ctop, face_flux_f32<DIR>(A, geomf, PL, zl, F, i, jf, kf, c));
#pragma unroll
      for (int v = 0; v < NV; v++) PL[v] = zh[v];
    }
  }
  warp_block_max(ctop, &A.clk->ctop_bits[DIR]);
}

}  // namespace grmhd
