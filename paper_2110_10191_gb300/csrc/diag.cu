// diag.cu -- the divergence diagnostic: the corner-centred divergence of
// sqrt(-g) B that flux-CT (Toth 2000; paper, "Implementation Notes", first
// paragraph) keeps at round-off.  At the corner shared by zones i-1..i,
// j-1..j, k-1..k:
//   div = sum_d [sum of sqrt(-g) B^d over the 4 zones on the + side of the
//          corner along d - the same over the 4 on the - side] / (4 dX_d)
// over directions with more than one zone; corners between interior zones
// only (a direction with one zone takes its single layer and the ghost copy
// below it).  Also the step's reciprocal, reciprocal square root and square
// root, and the bounds' quotients, on an array (grmhd_arith), so that their
// accuracy can be checked on the device.
#include "../../include/grmhd.h"
#include "grmhd_dev.cuh"
#include "grmhd_impl.h"
#include "step_bodies.cuh"

namespace grmhd {

__global__ void k_divb(StepArgs A, const double *__restrict__ P, unsigned long long *out) {
  const Dims &D = A.D;
  int lo[3], ext[3];
  for (int d = 0; d < 3; d++) {
    lo[d] = (D.n[d] > 1) ? NG + 1 : NG;
    ext[d] = (D.n[d] > 1) ? D.n[d] - 1 : 1;
  }
  const long long nc = (long long)ext[0] * ext[1] * ext[2];
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double div = 0.0, gb = 0.0;
  if (t < nc) {
    const int i = lo[0] + (int)(t % ext[0]);
    const int j = lo[1] + (int)((t / ext[0]) % ext[1]);
    const int k = lo[2] + (int)(t / ((long long)ext[0] * ext[1]));
    const double *gd = A.geom + (LOC_CENT * G_NCOMP + G_GDET) * D.n2d;
    for (int d = 0; d < 3; d++) {
      if (D.n[d] <= 1) continue;
      double sum = 0.0;
      for (int dk = -1; dk <= 0; dk++)
        for (int dj = -1; dj <= 0; dj++)
          for (int di = -1; di <= 0; di++) {
            const int side = (d == 0) ? di : (d == 1) ? dj : dk;  // 0: + side, -1: - side
            const long long z = zid(D, i + di, j + dj, k + dk);
            const double v = gd[(long long)(j + dj) * D.s[0] + (i + di)] * P[(B1 + d) * D.ntot + z];
            sum += side == 0 ? v : -v;
            gb = fmax(gb, fabs(v));
          }
      div += sum * (0.25 * A.idx[d]);
    }
  }
  warp_block_max(fabs(div), out);
  __syncthreads();  // both maxima use the same shared scratch
  warp_block_max(gb, out + 1);
}

void launch_divb(const StepArgs &A, const double *P, unsigned long long *out, cudaStream_t st) {
  long long nc = 1;
  for (int d = 0; d < 3; d++) nc *= (A.D.n[d] > 1) ? A.D.n[d] - 1 : 1;
  cudaMemsetAsync(out, 0, 2 * sizeof(unsigned long long), st);
  k_divb<<<(unsigned)((nc + BS - 1) / BS), BS, 0, st>>>(A, P, out);
}

}  // namespace grmhd

// ---------------------------------------------------------------------------
// The step's reciprocal, reciprocal square root and square root (rcp_nr,
// rsqrt_nr, sqrt_nr) on an array, so that their accuracy can be checked
// against the IEEE operations on the device.
// ---------------------------------------------------------------------------
namespace grmhd {

template <int FN>
__global__ void k_arith(const double *__restrict__ x, double *__restrict__ out, long long n) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double v = x[t];
  out[t] = FN == 0   ? rcp_nr(v)
           : FN == 1 ? rsqrt_nr(v)
           : FN == 2 ? sqrt_nr(v)
           : FN == 3 ? div_rn(v, FL_SIGMA, FL_SIGMA_RCP)
                     : div_rn(v, FL_TEMP, FL_TEMP_RCP);
}

}  // namespace grmhd

extern "C" int grmhd_arith(int fn, const double *x, double *out, long long n, void *stream) {
  if (fn < 0 || fn > 4 || n < 0 || (n > 0 && (!x || !out))) return GRMHD_ERR_INVALID;
  if (n == 0) return GRMHD_OK;
  const long long nb = (n + grmhd::BS - 1) / grmhd::BS;
  if (nb >= (1ll << 31)) return GRMHD_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  if (fn == 0) grmhd::k_arith<0><<<(unsigned)nb, grmhd::BS, 0, st>>>(x, out, n);
  if (fn == 1) grmhd::k_arith<1><<<(unsigned)nb, grmhd::BS, 0, st>>>(x, out, n);
  if (fn == 2) grmhd::k_arith<2><<<(unsigned)nb, grmhd::BS, 0, st>>>(x, out, n);
  if (fn == 3) grmhd::k_arith<3><<<(unsigned)nb, grmhd::BS, 0, st>>>(x, out, n);
  if (fn == 4) grmhd::k_arith<4><<<(unsigned)nb, grmhd::BS, 0, st>>>(x, out, n);
  return cudaGetLastError() == cudaSuccess ? GRMHD_OK : GRMHD_ERR_CUDA;
}
