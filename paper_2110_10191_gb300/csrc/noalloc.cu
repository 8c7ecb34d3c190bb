// noalloc.cu -- the face-flux stage for callers that cannot allocate device
// memory.
//
// Some callers cannot call cudaMalloc: code that runs while a memory pool is
// exhausted or frozen (a serving process that has pre-reserved all of HBM
// for simulation state), code inside frameworks whose allocator must not be
// bypassed, and host threads that may not trigger allocation while other
// work is being captured.  grmhd_fluxes_noalloc() gives them the flux stage
// of the step (reconstruction + local Lax-Friedrichs fluxes, boundary flux
// fixes, flux-CT) on buffers they already own, and keeps every intermediate
// (the metric at centres and faces, the edge EMFs, the signal-speed maxima)
// in one file-scope device array of fixed size instead of allocating it.
//
// The array is part of the library's device image: every GPU on which the
// library's kernels are loaded holds it (NOALLOC_SCRATCH_BYTES) until the
// process exits.  All calls share it and it keeps the last call's contents,
// so calls that overlap on the GPU (on different streams, or from different
// host threads) race on it; serialise them.
#include <cstddef>
#include <cstring>
#include <mutex>

#include "../../include/grmhd.h"
#include "grmhd_dev.cuh"
#include "grmhd_impl.h"
#include "sim_impl.h"

using namespace grmhd;

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(64) << 20;  // 64 MiB
constexpr int MAX_DEVICES = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device, looked up once per device
// (with that device current).  In host code the symbol itself is only a
// host-side stand-in, never a device address.  The table is guarded by a
// mutex: calls may come from several host threads.  An entry is dropped
// when a call on its device meets a CUDA error, so that after a device
// reset (which reloads the module, possibly at another address) the next
// call looks the address up again.
unsigned char *g_scratch_ptr[MAX_DEVICES];
std::mutex g_scratch_mu;

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

int scratch_for_current_device(int *dev_out, unsigned char **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GRMHD_ERR_CUDA;
  if (dev < 0 || dev >= MAX_DEVICES) return GRMHD_ERR_INVALID;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GRMHD_ERR_CUDA;
    g_scratch_ptr[dev] = (unsigned char *)p;
  }
  *dev_out = dev;
  *out = g_scratch_ptr[dev];
  return GRMHD_OK;
}

void forget_scratch(int dev) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  g_scratch_ptr[dev] = nullptr;
}

// Byte offsets of the pieces carved from the scratch for a grid of
// dimensions D: clock, geometry (3 locations), connection, bound
// thresholds, EMFs; off[5] is the total need.
void carve(const Dims &D, size_t off[6]) {
  off[0] = 0;
  off[1] = align_up(off[0] + sizeof(Clock));
  off[2] = align_up(off[1] + sizeof(double) * NLOC * G_NCOMP * (size_t)D.n2d);
  off[3] = align_up(off[2] + sizeof(double) * C_NCOMP * (size_t)D.n2d);
  off[4] = align_up(off[3] + sizeof(double) * 2 * (size_t)D.n2d);
  off[5] = align_up(off[4] + sizeof(double) * 3 * (size_t)D.ntot);
}

}  // namespace

extern "C" int grmhd_fluxes_noalloc(const grmhd_grid *grid, const grmhd_metric *metric,
                                    const grmhd_params *params, const double *P, double *F,
                                    double *ctop, void *stream) {
  if (!P || !F) return GRMHD_ERR_INVALID;
  Dims D;
  int rc = validate_problem(grid, metric, params, &D);  // the checks of grmhd_create
  if (rc != GRMHD_OK) return rc;
  const int n[3] = {grid->n1, grid->n2, grid->n3};
  const double xmin[3] = {grid->x1min, grid->x2min, grid->x3min};
  const double xmax[3] = {grid->x1max, grid->x2max, grid->x3max};
  size_t off[6];
  carve(D, off);
  if (off[5] > NOALLOC_SCRATCH_BYTES) return GRMHD_ERR_INVALID;  // grid too large for the scratch
  const size_t off_clk = off[0], off_geom = off[1], off_conn = off[2], off_floors = off[3],
               off_emf = off[4];

  int dev = 0;
  unsigned char *base = nullptr;
  rc = scratch_for_current_device(&dev, &base);
  if (rc != GRMHD_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  Clock *clk = (Clock *)(base + off_clk);

  GeomArgs G;
  G.D = D;
  G.kind = metric->kind;
  G.a = metric->a;
  G.h = metric->hslope;
  G.gam = params->gamma;
  for (int d = 0; d < 3; d++) {
    G.xmin[d] = xmin[d];
    G.dx[d] = (xmax[d] - xmin[d]) / n[d];
  }
  G.off[0] = G.off[1] = G.off[2] = 0;
  G.geom = (double *)(base + off_geom);
  G.conn = (double *)(base + off_conn);
  G.floors = (double *)(base + off_floors);

  StepArgs A;
  memset(&A, 0, sizeof(A));
  A.D = D;
  A.gam = params->gamma;
  A.igam = 1.0 / params->gamma;
  A.gm1 = params->gamma - 1.0;
  A.ggm1 = params->gamma * (params->gamma - 1.0);
  A.cfl = params->cfl;
  for (int d = 0; d < 3; d++) {
    A.dx[d] = G.dx[d];
    A.idx[d] = 1.0 / G.dx[d];
  }
  A.recon = params->recon;
  A.floors_on = params->floors_on;
  for (int d = 0; d < 3; d++)
    for (int sd = 0; sd < 2; sd++) A.bc[d][sd] = params->bc[d][sd];
  A.geom = G.geom;
  A.conn = G.conn;
  A.floors = G.floors;
  A.clk = clk;
  set_ff_constants(A);
  set_gas_constants(A);

  // faces outside the computed ranges read as zero, as in grmhd_get_fluxes
  const size_t fbytes = sizeof(double) * NV * (size_t)D.ntot;
  if (cudaMemsetAsync(F, 0, 3 * fbytes, st) != cudaSuccess) {
    forget_scratch(dev);
    return GRMHD_ERR_CUDA;
  }
  launch_geometry(G, st);
  launch_ctop_reset(A, st);
  double *Fd[3] = {F, F + NV * D.ntot, F + 2 * NV * D.ntot};
  launch_fluxes(A, P, Fd, st);
  launch_fix_ct(A, Fd, (double *)(base + off_emf), st);
  if (cudaGetLastError() != cudaSuccess) {
    forget_scratch(dev);
    return GRMHD_ERR_CUDA;
  }
  if (ctop) {
    unsigned long long bits[3];
    const void *src = (const unsigned char *)clk + offsetof(Clock, ctop_bits);
    if (cudaMemcpyAsync(bits, src, sizeof(bits), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      forget_scratch(dev);
      return GRMHD_ERR_CUDA;
    }
    for (int d = 0; d < 3; d++) memcpy(&ctop[d], &bits[d], sizeof(double));
  }
  return GRMHD_OK;
}
