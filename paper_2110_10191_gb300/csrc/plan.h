// plan.h -- the launch plan of the step over one or more grids (host side).
//
// Every grid of the step, whether a simulation stepped alone or a member of
// a batch, is advanced by the same plan kernels (plan.cu): one launch per
// kernel of the stage covers every grid of the plan, each block works on one
// grid, found through a per-class block -> grid table, and runs the per-thread
// body of step_bodies.cuh / mixed_bodies.cuh for its thread index within that
// grid.  Since the machine code is the same whatever the plan holds, a
// grid's results are bitwise independent of the grids it is stepped with.
#pragma once

#include <cuda_runtime.h>

#include "grmhd_impl.h"

namespace grmhd {

// One grid as the plan kernels see it.
struct StageItem {
  StepArgs A;
  double *P, *Ph;  // stage arrays: P^n / P^{n+1} and P^{n+1/2}
  double *F[3], *emf, *Lf, *Rf, *Uc;
  int *pflag, *fflag;
  float *Pf;           // mixed precision: FP32 primitives (8 x ntot)
  const float *geomf;  // mixed precision: FP32 geometry
  int mixed;           // 1: FP32 flux stage
};

// launch classes, each with its own block table
enum {
  PC_BX1,
  PC_BX2,
  PC_BX3,
  PC_RECON01,  // FP64 reconstruction along X1 and X2
  PC_RECON2,   // along X3 (none for flat-X3 grids)
  PC_FACE0,
  PC_FACE1,
  PC_FACE2,
  PC_TOF32,  // mixed: FP32 copy of the stage input
  PC_RECON01F,
  PC_RECON2F,
  PC_FACE0F,
  PC_FACE1F,
  PC_FACE2F,
  PC_REPL,  // flat-X3 flux copies
  PC_FIX,
  PC_EDGE,  // EMFs and CT
  PC_ZONE,  // update and fixup
  PC_N
};

struct Plan {
  int ngrid;
  StageItem *items;  // device
  int *tab;          // device: per class, ngrid + 1 first blocks, then the block -> grid map
  int off_base[PC_N], map_base[PC_N], nblocks[PC_N];
  long long zones;  // interior zones over all grids
};

// Observer of the launches, per kernel class GRMHD_K_* (profiling).
struct PlanHook {
  virtual void begin(int kclass, int nlaunch) = 0;
  virtual void end(int kclass) = 0;
  virtual ~PlanHook() {}
};

// Build the tables and upload the items (device memory of the plan);
// GRMHD_OK, GRMHD_ERR_INVALID (more than 2^31 - 1 blocks in a launch),
// GRMHD_ERR_NOMEM or GRMHD_ERR_CUDA.
int plan_build(Plan &p, const StageItem *items, int n);
void plan_free(Plan &p);

// The functions below enqueue on st and return the number of kernels
// launched; launch errors are left for cudaGetLastError().
// stage input: 0 = P, 1 = Ph.  Signal-speed reset, reconstruction + face
// fluxes (FP64 or FP32 per grid), flat-X3 copies.
int plan_fluxes(const Plan &p, int in, cudaStream_t st, PlanHook *h);
// per-grid clock: 0 reset the signal-speed maxima, 1 CFL time step, 2 advance
int plan_clock(const Plan &p, int op, cudaStream_t st, PlanHook *h);
// boundary flux fixes + flux-CT
int plan_fix_ct(const Plan &p, cudaStream_t st, PlanHook *h);
// U(P) + dtfac dt (S(in) - div F) -> inversion -> bounds into the other array
// (in 0: P -> Ph, in 1: Ph -> P), then the fixup; ucache_mode as launch_update
int plan_update(const Plan &p, int in, double dtfac, int ucache_mode, cudaStream_t st, PlanHook *h);
// ghost fill of P (which 0) or Ph (which 1)
int plan_bounds(const Plan &p, int which, cudaStream_t st, PlanHook *h);
// one stage: stage 0 predictor (P -> Ph, dt/2, with the CFL step),
// stage 1 corrector (Ph -> P, dt)
int plan_stage(const Plan &p, int stage, int ucache_mode, cudaStream_t st, PlanHook *h);
// full predictor-corrector steps (U(P^n) kept between the stages)
int plan_steps(const Plan &p, int nsteps, cudaStream_t st, PlanHook *h);

}  // namespace grmhd
