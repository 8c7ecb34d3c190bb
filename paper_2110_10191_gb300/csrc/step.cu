// step.cu -- the single-grid kernels of the allocation-free flux entry
// point (noalloc.cu): fused reconstruction + LLF face fluxes, the
// signal-speed reset, the boundary flux fixes and flux-CT; and the
// interior <-> ghost layout copies.  The step itself runs the plan kernels
// (plan.cu) on the same per-thread bodies (step_bodies.cuh).
#include "grmhd_dev.cuh"
#include "grmhd_impl.h"
#include "step_bodies.cuh"

namespace grmhd {

__device__ __forceinline__ long long gtid() { return blockIdx.x * (long long)blockDim.x + threadIdx.x; }

static unsigned nblk(long long n) { return (unsigned)((n + BS - 1) / BS); }

// ---------------------------------------------------------------------------
// Fused face fluxes (reconstruction and LLF in one pass per face; used by
// the allocation-free flux entry point, which has no room for the face-value
// scratch of the split stage).  Face box for direction d: d-index NG .. n_d+NG,
// transverse NG-1 .. n_e+NG.
// ---------------------------------------------------------------------------
template <int DIR, int RECON>
__global__ void __launch_bounds__(BS) k_flux(StepArgs A, const double *__restrict__ P,
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
    double PL[NV], PR[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) {
      const double *p = P + v * D.ntot + c;
      if (RECON == 1) {
        const double x0 = __ldg(p - 3 * st), x1 = __ldg(p - 2 * st), x2 = __ldg(p - st);
        const double x3 = __ldg(p), x4 = __ldg(p + st), x5 = __ldg(p + 2 * st);
        PL[v] = weno5_hi(x0, x1, x2, x3, x4);
        PR[v] = weno5_hi(x5, x4, x3, x2, x1);
      } else {
        const double x1 = __ldg(p - 2 * st), x2 = __ldg(p - st);
        const double x3 = __ldg(p), x4 = __ldg(p + st);
        PL[v] = x2 + 0.5 * mc_slope(x1, x2, x3);
        PR[v] = x3 - 0.5 * mc_slope(x2, x3, x4);
      }
    }
    const int loc = (DIR == 0) ? LOC_FACE1 : (DIR == 1) ? LOC_FACE2 : LOC_CENT;
    Geo G;
    load_geo(A.geom + (long long)loc * G_NCOMP * D.n2d, D.n2d, (long long)j * D.s[0] + i, G);
    FState sL, sR;
    fluid_state(PL, G, sL);
    fluid_state(PR, G, sR);
    const double ct = fmax(mhd_cmax(PL, sL, G, A.gam, A.ggm1, DIR + 1),
                           mhd_cmax(PR, sR, G, A.gam, A.ggm1, DIR + 1));
    double FL[NV], FR[NV], UL[NV], UR[NV];
    prim_flux(PL, sL, G, A.gam, DIR + 1, FL);
    prim_flux(PR, sR, G, A.gam, DIR + 1, FR);
    prim_flux(PL, sL, G, A.gam, 0, UL);
    prim_flux(PR, sR, G, A.gam, 0, UR);
#pragma unroll
    for (int v = 0; v < NV; v++) F[v * D.ntot + c] = 0.5 * (FL[v] + FR[v] - ct * (UR[v] - UL[v]));
    bool interior = true;
#pragma unroll
    for (int e = 0; e < 3; e++) {
      if (e == DIR) continue;
      const int q = (e == 0) ? i : (e == 1) ? j : k;
      interior = interior && (q >= NG) && (q < D.n[e] + NG);
    }
    if (interior) ctop = ct;
  }
  warp_block_max(ctop, &A.clk->ctop_bits[DIR]);
}

template <int DIR>
static void launch_flux_dir(const StepArgs &A, const double *P, double *F, cudaStream_t st) {
  const Dims &D = A.D;
  long long nf = 1;
  for (int e = 0; e < 3; e++) nf *= (e == DIR) ? D.n[e] + 1 : D.n[e] + 2;
  if (A.recon == 1)
    k_flux<DIR, 1><<<nblk(nf), BS, 0, st>>>(A, P, F);
  else
    k_flux<DIR, 0><<<nblk(nf), BS, 0, st>>>(A, P, F);
}

void launch_fluxes(const StepArgs &A, const double *P, double *F[3], cudaStream_t st) {
  launch_flux_dir<0>(A, P, F[0], st);
  launch_flux_dir<1>(A, P, F[1], st);
  launch_flux_dir<2>(A, P, F[2], st);
}

__global__ void k_reset_ctop(Clock *clk) { reset_ctop_body(clk); }

void launch_ctop_reset(const StepArgs &A, cudaStream_t st) { k_reset_ctop<<<1, 1, 0, st>>>(A.clk); }

// ---------------------------------------------------------------------------
// Boundary flux fixes and flux-CT
// ---------------------------------------------------------------------------
__global__ void k_fix_flux(StepArgs A, double *F1, double *F2) {
  fix_flux_body(A, F1, F2, nullptr, nullptr, gtid());
}

__global__ void k_emf(StepArgs A, const double *__restrict__ F1, const double *__restrict__ F2,
                      const double *__restrict__ F3, double *__restrict__ emf) {
  emf_body(A, F1, F2, F3, emf, gtid());
}

__global__ void k_ct(StepArgs A, double *F1, double *F2, double *F3, const double *__restrict__ emf) {
  ct_body(A, F1, F2, F3, emf, gtid());
}

void launch_fix_ct(const StepArgs &A, double *F[3], double *emf, cudaStream_t st) {
  const Dims &D = A.D;
  k_fix_flux<<<nblk(n_fix(D)), BS, 0, st>>>(A, F[0], F[1]);
  k_emf<<<nblk(n_edge(D)), BS, 0, st>>>(A, F[0], F[1], F[2], emf);
  k_ct<<<nblk(n_edge(D)), BS, 0, st>>>(A, F[0], F[1], F[2], emf);
}

// ---------------------------------------------------------------------------
// Interior <-> ghost layout copies
// ---------------------------------------------------------------------------
__global__ void k_pack(Dims D, const double *__restrict__ src, double *__restrict__ dst,
                       int to_ghost, int nvar) {
  const long long nz = (long long)D.n[0] * D.n[1] * D.n[2];
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= nz * nvar) return;
  const long long v = t / nz, r = t % nz;
  const int i = (int)(r % D.n[0]);
  const int j = (int)((r / D.n[0]) % D.n[1]);
  const int k = (int)(r / ((long long)D.n[0] * D.n[1]));
  const long long g = v * D.ntot + zid(D, i + NG, j + NG, k + NG);
  if (to_ghost)
    dst[g] = src[t];
  else
    dst[t] = src[g];
}

void launch_pack(const Dims &D, const double *src, double *dst, int to_ghost, cudaStream_t st,
                 int nvar) {
  const long long n = (long long)D.n[0] * D.n[1] * D.n[2] * nvar;
  k_pack<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(D, src, dst, to_ghost, nvar);
}

}  // namespace grmhd
