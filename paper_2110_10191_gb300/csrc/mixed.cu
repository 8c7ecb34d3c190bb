// mixed.cu -- geometry copies for the reduced-word flux stages: the FP32
// copy (mixed-precision mode) and the split float-float copy (float-float
// mode) of a simulation's geometry, built once and again when the geometry
// is replaced.  The flux-stage kernels themselves are plan kernels (plan.cu).
#include "grmhd_impl.h"
#include "ff_bodies.cuh"
#include "mixed_bodies.cuh"

namespace grmhd {

__global__ void k_to_f32(long long n, const double *__restrict__ src, float *__restrict__ dst) {
  to_f32_body(src, dst, n, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

void launch_to_f32(long long n, const double *src, float *dst, cudaStream_t st) {
  k_to_f32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, src, dst);
}

__global__ void k_to_ff(long long n, const double *__restrict__ src, float *__restrict__ dst) {
  to_ff_body(src, dst, n, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

void launch_to_ff(long long n, const double *src, float *dst, cudaStream_t st) {
  k_to_ff<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, src, dst);
}

}  // namespace grmhd
