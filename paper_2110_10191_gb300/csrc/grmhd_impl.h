// grmhd_impl.h -- kernel argument blocks and launch entry points shared by
// the translation units of the library (host side).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "grmhd_dev.cuh"

namespace grmhd {

struct GeomArgs {
  Dims D;
  int kind;
  double a, h, gam;
  double xmin[3], dx[3];
  double *geom;    // [NLOC][G_NCOMP][n2d]
  double *conn;    // [C_NCOMP][n2d]
  double *floors;  // [2][n2d]
};

// Device-resident clock of a simulation (updated by kernels only, so a
// whole step can be enqueued or captured without a host round trip).
struct Clock {
  double t, dt, dt_prev, t_final;
  long long steps;
  unsigned long long ctop_bits[3];  // max signal speed per direction (as bits, >= 0)
  unsigned long long counters[4];   // inversion failures, floor hits, unrecoverable, spare
};

struct StepArgs {
  Dims D;
  double gam, igam, cfl;  // adiabatic index, its reciprocal, Courant number
  double dx[3], idx[3];  // zone widths and their reciprocals
  int recon, floors_on;
  int bc[3][2];
  const double *geom;
  const double *conn;
  const double *floors;
  Clock *clk;
};

void launch_geometry(const GeomArgs &A, cudaStream_t st);

// boundary conditions on a primitive set
void launch_bounds(const StepArgs &A, double *P, cudaStream_t st);
// zero clk->ctop_bits before a flux pass
void launch_ctop_reset(const StepArgs &A, cudaStream_t st);
// fluxes of P (recon + LLF), with the interior ctop maxima into clk->ctop_bits
void launch_fluxes(const StepArgs &A, const double *P, double *F[3], cudaStream_t st);
// the same fluxes in two passes per direction: zone-centric reconstruction of
// both face values of every zone along dir into Lf (low face) / Rf (high face),
// scratch of 8 x ntot doubles each, then the face fluxes from them
void launch_recon(const StepArgs &A, int dir, const double *P, double *Lf, double *Rf,
                  cudaStream_t st);
void launch_face(const StepArgs &A, int dir, double *F, const double *Lf, const double *Rf,
                 cudaStream_t st);
// mixed precision: FP32 copies and the FP32 flux stage (fluxes written in FP64)
void launch_to_f32(long long n, const double *src, float *dst, cudaStream_t st);
void launch_recon_f32(const StepArgs &A, int dir, const float *P, float *Lf, float *Rf,
                      cudaStream_t st);
void launch_face_f32(const StepArgs &A, int dir, const float *geomf, double *F, const float *Lf,
                     const float *Rf, cudaStream_t st);
// time step from clk->ctop_bits (stage 1 only)
void launch_dt(const StepArgs &A, cudaStream_t st);
// boundary flux fixes + flux-CT (emf scratch: 3 x ntot)
void launch_fix_ct(const StepArgs &A, double *F[3], double *emf, cudaStream_t st);
// U(Pi) + dt' (S(Ps) - div F) -> invert -> floors; dtfac 0.5 (predictor) or 1;
// ucache_mode 1: store U(Pi) in Ucache (needs Ps == Pi), 2: read U(Pi) from it,
// 0: neither
void launch_update(const StepArgs &A, const double *Pi, const double *Ps, double *Pout,
                   double *const F[3], int *pflag, int *fflag, double dtfac, double *Ucache,
                   int ucache_mode, cudaStream_t st);
void launch_fixup(const StepArgs &A, double *Pout, const int *pflag, int *fflag, cudaStream_t st);
// t += dt, steps++ (when dt > 0)
void launch_advance(const StepArgs &A, cudaStream_t st);
// pack interior <-> ghost layout
void launch_pack(const Dims &D, const double *src, double *dst, int to_ghost, cudaStream_t st);

}  // namespace grmhd
