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
  float *Pff;          // float-float: split primitives ([2][8][ntot])
  const float *geomff; // float-float: split geometry ([2][NLOC][G_NCOMP][n2d])
  int prec;            // GRMHD_PREC_*: the flux stage's arithmetic
  // electrons (A.elec): (kappa_tot, kappa_e) of the stage arrays ([2][ntot]
  // each, with P and Ph), their fluxes, and U_rho(P^n) kept by the predictor
  double *K, *Kh, *FK[3], *Uek;
  double *KLf, *KRf;  // their face values along the current direction
};

// launch classes, each with its own block table
enum {
  PC_BX1,
  PC_BX2,
  PC_BX3,
  PC_RECON0,  // FP64 reconstruction along X1 (column walks)
  PC_RECON1,  // along X2
  PC_RECON2,  // along X3 (none for flat-X3 grids)
  PC_FACE0,
  PC_FACE1,
  PC_FACE2,
  PC_FACE0E,  // FP64 face fluxes of grids with electrons (they also store the entropy weights)
  PC_FACE1E,
  PC_FACE2E,
  PC_TOF32,  // mixed: FP32 copy of the stage input
  PC_FACE0F, // mixed: fused FP32 reconstruction + face fluxes per direction
  PC_FACE1F,
  PC_FACE2F,
  PC_TOFF,  // float-float: split copy of the stage input
  PC_RECON01X,
  PC_RECON2X,
  PC_FACE0X,
  PC_FACE1X,
  PC_FACE2X,
  PC_REPL,  // flat-X3 flux copies
  PC_FIX,
  PC_EDGE,   // EMFs and CT
  PC_ZONE,   // fixup (every grid)
  PC_UPD64,  // FP64 update (FP64 and mixed-precision grids)
  PC_UPDX,   // float-float update (float-float and mixed + float-float grids)
  PC_FLOORD, // drift-frame bounds (grids with bounds in the drift frame, no electrons)
  PC_EREC01, // electron entropy reconstruction along X1, X2 (grids with electrons)
  PC_EREC2,  // along X3
  PC_EFACE0, // electron entropy fluxes per direction
  PC_EFACE1,
  PC_EFACE2,
  PC_EZONE,  // electron heating + bounds, and their fixup (grids with electrons)
  PC_N
};

// block order of a launch class
enum {
  PLAN_SCHED_GRID = 0,  // grids in plan order, each grid's blocks contiguous
  PLAN_SCHED_LPT = 1,   // grids by decreasing block count (largest first), contiguous
  PLAN_SCHED_RR = 2,    // round robin: one block of each grid that has blocks left, in turn
  PLAN_SCHED_N
};

struct Plan {
  int ngrid;
  StageItem *items;  // device
  StageItem *host_items;  // host copy of items
  int *tab;          // device: per class, the grid of each block, then its index within that grid
  long long tab_cap; // ints allocated for tab (enough for 64-thread blocks in every class)
  long long *count;  // host: threads of each grid per class, [PC_N][ngrid]
  int bs[PC_N];      // threads per block of each class (multiple of 32, <= 256)
  int sched[PC_N];   // block order of each class (SCHED_*)
  int map_base[PC_N], loc_base[PC_N], nblocks[PC_N];
  long long zones;  // interior zones over all grids
  int tuned;        // 1 after plan_autotune
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
// threads per launch class of one grid (dimensions, flat X3, GRMHD_PREC_*,
// bounds in the drift frame, electrons evolved, the plan's reconstruction
// walk length)
void plan_counts(const Dims &D, int flat3, int prec, int drift, int elec, int rwalk,
                 long long c[PC_N]);
// The FP64 reconstruction's walk length for a plan of these grids: the
// longest of 16, 8, 4, 2 zones per thread that still gives each of its
// launches RWALK_MIN_THREADS threads, else 1 (one thread per zone).  About
// 20 warps per SM keep the FP64 unit at its issue rate; with fewer, each
// thread's longer chain of dependent work shows (64 small 2D grids with
// 2-zone walks, 11 warps per SM: 115 us per launch against 84 us one
// thread per zone).
constexpr long long RWALK_MIN_THREADS = 152 * 640;
int plan_rwalk(const StageItem *items, int n);
// Set the plan's reconstruction walk length (1, 2, 4, 8 or 16 zones per
// thread; 0: plan_rwalk's choice) and re-lay the reconstruction's block
// tables.  The values do not depend on it.
int plan_set_rwalk(Plan &p, int rw);
// device bytes a one-grid plan of such a grid holds (item + block tables)
long long plan_bytes(const Dims &D, int flat3, int prec, int drift, int elec);
void plan_free(Plan &p);
// Re-lay the block tables of class cls for bs threads per block and block
// order sched (the results of every grid do not depend on either).
int plan_set_class(Plan &p, int cls, int bs, int sched);
// Pick, by timing on st, the block size and block order of each heavy
// launch class (reconstruction, face fluxes, update + fixup, in both
// precisions) among 64/128/256 threads and the SCHED_* orders.  Leaves
// every grid's state and clock as it found them: the trial launches write
// only scratch (face values, fluxes, the interior of the half-step array)
// and the failure/bound flags of the last stage, and the clocks are saved
// and restored.  Waits for the device before and after.  ms_before / ms_after (may be NULL): one
// pass of the tuned kernels with the previous and the chosen settings.
int plan_autotune(Plan &p, int trials, cudaStream_t st, double *ms_before, double *ms_after);

// The functions below enqueue on st and return the number of kernels
// launched; launch errors are left for cudaGetLastError().
// stage input: 0 = P, 1 = Ph.  Signal-speed reset, reconstruction + face
// fluxes (FP64, FP32 or float-float per grid), flat-X3 copies.
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
// the pieces of plan_update and plan_bounds, for a decomposed grid that
// exchanges block edges between them: the update alone (into 1 - in), the
// fixup of array out, one ghost-fill pass (0: X1, 1: X2, 2: X3)
int plan_update_only(const Plan &p, int in, double dtfac, int ucache_mode, cudaStream_t st,
                     PlanHook *h);
int plan_fixup(const Plan &p, int out, cudaStream_t st, PlanHook *h);
int plan_bounds_pass(const Plan &p, int which, int pass, cudaStream_t st, PlanHook *h);
// one stage: stage 0 predictor (P -> Ph, dt/2, with the CFL step),
// stage 1 corrector (Ph -> P, dt)
int plan_stage(const Plan &p, int stage, int ucache_mode, cudaStream_t st, PlanHook *h);
// full predictor-corrector steps (U(P^n) kept between the stages)
int plan_steps(const Plan &p, int nsteps, cudaStream_t st, PlanHook *h);

}  // namespace grmhd
