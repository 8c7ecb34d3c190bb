// probe.cu -- measured double-precision throughput of the current GPU, the
// peak against which the FP64-bound kernels of the step are reported.
//
// grmhd_fp64_peak: every thread runs 8 independent dependent-FMA chains (the
// pipe is fed without waiting on latency) on a grid that is a multiple of
// the SM count; FLOP/s from CUDA events.
// grmhd_fp64_probe: the same loop for a chosen operation (FMA, add,
// multiply), number of chains and blocks per SM, with the SM clock measured
// inside the kernel (clock64 against the global nanosecond timer), so that
// the FP64 issue rate comes out per SM and per clock cycle whatever clock
// the GPU ran at.
#include <cuda_runtime.h>

#include "../../include/grmhd.h"

namespace {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// OP 0: a = a m + c (FMA); 1: a = a + c; 2: a = a m.  tim (may be null):
// per block, SM cycles and nanoseconds between thread 0's start and end.
template <int CH, int OP>
__global__ void k_fp64(long long iters, double seed, double *sink, unsigned long long *tim) {
  double a[CH];
#pragma unroll
  for (int q = 0; q < CH; q++) a[q] = seed + threadIdx.x + q;
  const double m = 0.999999999, c = 1e-9;
  unsigned long long c0 = 0, g0 = 0;
  if (tim && threadIdx.x == 0) {
    c0 = clock64();
    g0 = global_ns();
  }
  for (long long i = 0; i < iters; i++) {
#pragma unroll
    for (int q = 0; q < CH; q++) {
      if (OP == 0) a[q] = fma(a[q], m, c);
      if (OP == 1) a[q] = a[q] + c;
      if (OP == 2) a[q] = a[q] * m;
    }
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < CH; q++) s += a[q];
  if (s == 12345.678) sink[blockIdx.x] = s;  // keeps the chains live
  if (tim && threadIdx.x == 0) {
    tim[2 * blockIdx.x] = clock64() - c0;
    tim[2 * blockIdx.x + 1] = global_ns() - g0;
  }
}

using KFn = void (*)(long long, double, double *, unsigned long long *);

template <int OP>
KFn pick(int chains) {
  switch (chains) {
    case 1: return k_fp64<1, OP>;
    case 2: return k_fp64<2, OP>;
    case 4: return k_fp64<4, OP>;
    case 8: return k_fp64<8, OP>;
    case 16: return k_fp64<16, OP>;
  }
  return nullptr;
}

// Runs k on blocks x threads once to warm up and once timed; ms from CUDA
// events, and (tim != null) the mean SM cycles and nanoseconds of the blocks.
int timed_run(KFn k, int blocks, int threads, long long iters, double *ms_out, double *cyc_out,
              double *ns_out) {
  double *sink = nullptr;
  unsigned long long *tim = nullptr;
  if (cudaMalloc(&sink, sizeof(double) * blocks) != cudaSuccess) return GRMHD_ERR_NOMEM;
  if (cyc_out && cudaMalloc(&tim, sizeof(unsigned long long) * 2 * blocks) != cudaSuccess) {
    cudaFree(sink);
    return GRMHD_ERR_NOMEM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k<<<blocks, threads>>>(iters / 10 + 1, 1.0, sink, tim);  // warm-up
  cudaEventRecord(e0);
  k<<<blocks, threads>>>(iters, 1.0, sink, tim);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  int rc = (err == cudaSuccess && cudaGetLastError() == cudaSuccess) ? GRMHD_OK : GRMHD_ERR_CUDA;
  if (rc == GRMHD_OK && cyc_out) {
    unsigned long long *h = new unsigned long long[2 * (size_t)blocks];
    if (cudaMemcpy(h, tim, sizeof(unsigned long long) * 2 * blocks, cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      rc = GRMHD_ERR_CUDA;
    double cyc = 0.0, ns = 0.0;
    for (int b = 0; b < blocks; b++) {
      cyc += (double)h[2 * b];
      ns += (double)h[2 * b + 1];
    }
    delete[] h;
    *cyc_out = cyc / blocks;
    *ns_out = ns / blocks;
  }
  *ms_out = ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (tim) cudaFree(tim);
  return rc;
}

int sm_count(int *nsm) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GRMHD_ERR_CUDA;
  if (cudaDeviceGetAttribute(nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return GRMHD_ERR_CUDA;
  return GRMHD_OK;
}

}  // namespace

extern "C" int grmhd_fp64_peak(long long iters, double *flops) {
  if (!flops || iters < 1) return GRMHD_ERR_INVALID;
  int nsm = 0;
  int rc = sm_count(&nsm);
  if (rc != GRMHD_OK) return rc;
  const int threads = 256, blocks = nsm * 8;
  double ms = 0.0;
  rc = timed_run(k_fp64<8, 0>, blocks, threads, iters, &ms, nullptr, nullptr);
  if (rc != GRMHD_OK) return rc;
  *flops = 2.0 * 8.0 * (double)iters * threads * blocks / (ms * 1e-3);
  return GRMHD_OK;
}

extern "C" int grmhd_fp64_probe(int op, int chains, int blocks_per_sm, long long iters,
                                double *ops_per_sm_clock, double *sm_mhz) {
  if (!ops_per_sm_clock || !sm_mhz || iters < 1 || op < 0 || op > 2 || blocks_per_sm < 1 ||
      blocks_per_sm > 16)
    return GRMHD_ERR_INVALID;
  KFn k = op == 0 ? pick<0>(chains) : op == 1 ? pick<1>(chains) : pick<2>(chains);
  if (!k) return GRMHD_ERR_INVALID;
  int nsm = 0;
  int rc = sm_count(&nsm);
  if (rc != GRMHD_OK) return rc;
  const int threads = 128, blocks = nsm * blocks_per_sm;
  double ms = 0.0, cyc = 0.0, ns = 0.0;
  rc = timed_run(k, blocks, threads, iters, &ms, &cyc, &ns);
  if (rc != GRMHD_OK) return rc;
  if (!(ns > 0.0) || !(ms > 0.0)) return GRMHD_ERR_CUDA;
  const double mhz = cyc / ns * 1e3;
  const double ops = (double)chains * iters * threads * blocks;
  *sm_mhz = mhz;
  *ops_per_sm_clock = ops / (ms * 1e-3 * mhz * 1e6) / nsm;
  return GRMHD_OK;
}
