// probe.cu -- measured double-precision FMA throughput of the current GPU,
// the peak against which the FP64-bound kernels of the step are reported.
// Every thread runs 8 independent dependent-FMA chains, so the pipe is fed
// without waiting on latency; the grid is a multiple of the SM count.
#include <cuda_runtime.h>

#include "../../include/grmhd.h"

namespace {

__global__ void k_dfma(long long iters, double seed, double *sink) {
  double a0 = seed + threadIdx.x, a1 = a0 + 1.0, a2 = a0 + 2.0, a3 = a0 + 3.0;
  double a4 = a0 + 4.0, a5 = a0 + 5.0, a6 = a0 + 6.0, a7 = a0 + 7.0;
  const double m = 0.999999999, c = 1e-9;
  for (long long i = 0; i < iters; i++) {
    a0 = fma(a0, m, c); a1 = fma(a1, m, c); a2 = fma(a2, m, c); a3 = fma(a3, m, c);
    a4 = fma(a4, m, c); a5 = fma(a5, m, c); a6 = fma(a6, m, c); a7 = fma(a7, m, c);
  }
  const double s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (s == 12345.678) sink[blockIdx.x] = s;  // keeps the chains live
}

}  // namespace

extern "C" int grmhd_fp64_peak(long long iters, double *flops) {
  if (!flops || iters < 1) return GRMHD_ERR_INVALID;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GRMHD_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return GRMHD_ERR_CUDA;
  const int threads = 256, blocks = nsm * 8;
  double *sink = nullptr;
  if (cudaMalloc(&sink, sizeof(double) * blocks) != cudaSuccess) return GRMHD_ERR_NOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_dfma<<<blocks, threads>>>(iters / 10 + 1, 1.0, sink);  // warm-up
  cudaEventRecord(e0);
  k_dfma<<<blocks, threads>>>(iters, 1.0, sink);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (err != cudaSuccess || cudaGetLastError() != cudaSuccess) return GRMHD_ERR_CUDA;
  *flops = 2.0 * 8.0 * (double)iters * threads * blocks / (ms * 1e-3);
  return GRMHD_OK;
}
