// mixed.cu -- the flux stage of the mixed-precision mode.
//
// An FP32 copy of the primitives (with ghosts) and of the geometry feeds a
// zone-centric FP32 reconstruction and an FP32 face-flux kernel (fluid
// state, signal speeds, local Lax-Friedrichs flux); the fluxes are written
// in FP64, so the flux-CT EMF combination, the conserved-variable
// accumulation, the 1D_W inversion and the bounds run in FP64 as in the
// full-FP64 mode.  The signal-speed maxima for the time step come from the
// FP32 states.
#include <cfloat>

#include "grmhd_f32.cuh"
#include "grmhd_impl.h"

namespace grmhd {

constexpr int BSM = 128;

__global__ void k_to_f32(long long n, const double *__restrict__ src, float *__restrict__ dst) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double x = src[t];
  // clamp to the float range (metric components at the poles)
  dst[t] = (float)fmax(fmin(x, (double)FLT_MAX), -(double)FLT_MAX);
}

void launch_to_f32(long long n, const double *src, float *dst, cudaStream_t st) {
  k_to_f32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, src, dst);
}

template <int DIR, int RECON>
__global__ void __launch_bounds__(BSM) k_recon_f32(StepArgs A, const float *__restrict__ P,
                                                   float *__restrict__ Lf, float *__restrict__ Rf) {
  const Dims &D = A.D;
  const int e0 = D.n[0] + 2, e1 = D.n[1] + 2, e2 = D.n[2] + 2;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)e0 * e1 * e2) return;
  const int i = NG - 1 + (int)(t % e0);
  const int j = NG - 1 + (int)((t / e0) % e1);
  const int k = NG - 1 + (int)(t / ((long long)e0 * e1));
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

__device__ __forceinline__ void block_max_f64(double v, unsigned long long *dst) {
  unsigned long long b = __double_as_longlong(v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long x = __shfl_xor_sync(0xffffffffu, b, o);
    b = (x > b) ? x : b;
  }
  __shared__ unsigned long long sm[BSM / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sm[w] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = sm[0];
    for (int q = 1; q < BSM / 32; q++) m = (sm[q] > m) ? sm[q] : m;
    if (m) atomicMax(dst, m);
  }
}

template <int DIR>
__global__ void __launch_bounds__(BSM) k_face_f32(StepArgs A, const float *__restrict__ geomf,
                                                  const float *__restrict__ Lf,
                                                  const float *__restrict__ Rf,
                                                  double *__restrict__ F) {
  const Dims &D = A.D;
  int lo[3], ext[3];
#pragma unroll
  for (int e = 0; e < 3; e++) {
    lo[e] = (e == DIR) ? NG : NG - 1;
    ext[e] = (e == DIR) ? D.n[e] + 1 : D.n[e] + 2;
  }
  const long long nface = (long long)ext[0] * ext[1] * ext[2];
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
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
    bool interior = true;
#pragma unroll
    for (int e = 0; e < 3; e++) {
      if (e == DIR) continue;
      const int q = (e == 0) ? i : (e == 1) ? j : k;
      interior = interior && (q >= NG) && (q < D.n[e] + NG);
    }
    if (interior) ctop = (double)ct;
  }
  block_max_f64(ctop, &A.clk->ctop_bits[DIR]);
}

template <int DIR>
static void recon_f32_dir(const StepArgs &A, const float *P, float *Lf, float *Rf, cudaStream_t st) {
  const Dims &D = A.D;
  const long long nz = (long long)(D.n[0] + 2) * (D.n[1] + 2) * (D.n[2] + 2);
  const unsigned nb = (unsigned)((nz + BSM - 1) / BSM);
  if (A.recon == 1)
    k_recon_f32<DIR, 1><<<nb, BSM, 0, st>>>(A, P, Lf, Rf);
  else
    k_recon_f32<DIR, 0><<<nb, BSM, 0, st>>>(A, P, Lf, Rf);
}

template <int DIR>
static void face_f32_dir(const StepArgs &A, const float *geomf, double *F, const float *Lf,
                         const float *Rf, cudaStream_t st) {
  const Dims &D = A.D;
  long long nf = 1;
  for (int e = 0; e < 3; e++) nf *= (e == DIR) ? D.n[e] + 1 : D.n[e] + 2;
  k_face_f32<DIR><<<(unsigned)((nf + BSM - 1) / BSM), BSM, 0, st>>>(A, geomf, Lf, Rf, F);
}

void launch_recon_f32(const StepArgs &A, int dir, const float *P, float *Lf, float *Rf,
                      cudaStream_t st) {
  if (dir == 0) recon_f32_dir<0>(A, P, Lf, Rf, st);
  if (dir == 1) recon_f32_dir<1>(A, P, Lf, Rf, st);
  if (dir == 2) recon_f32_dir<2>(A, P, Lf, Rf, st);
}

void launch_face_f32(const StepArgs &A, int dir, const float *geomf, double *F, const float *Lf,
                     const float *Rf, cudaStream_t st) {
  if (dir == 0) face_f32_dir<0>(A, geomf, F, Lf, Rf, st);
  if (dir == 1) face_f32_dir<1>(A, geomf, F, Lf, Rf, st);
  if (dir == 2) face_f32_dir<2>(A, geomf, F, Lf, Rf, st);
}

}  // namespace grmhd
