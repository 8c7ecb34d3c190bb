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
  int off[3];      // global index of the first interior zone (blocks of a decomposed grid; else 0)
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

// boundary code of a side shared with another block of a decomposed grid:
// the bounds leave its ghosts to the exchange between blocks
constexpr int BC_EXCHANGE = 4;

struct StepArgs {
  Dims D;
  double gam, igam, cfl;  // adiabatic index, its reciprocal, Courant number
  double gm1, ggm1;       // gamma - 1 and gamma (gamma - 1)
  GasK gk;                // the inversion's and the bounds' constants (set_gas_constants)
  double dx[3], idx[3];  // zone widths and their reciprocals
  int recon, floors_on;
  // zones per thread of the FP64 reconstruction along a column (2..16), or 1:
  // one thread per zone; set by the plan from its grids' sizes
  int rwalk;
  int floor_drift;  // bounds in the drift frame: a separate pass after the update
  // electron entropies (GRMHD_ELEC_* model, 0: off): adiabatic indices of
  // electrons and protons, the constant share, the bounds on T_p/T_e
  int elec;
  double game, gamp, fel_const, tpte_min, tpte_max;
  // electrons: per face, the weights of the left and right entropies in
  // their LLF flux, [3][2][ntot] (direction, side)
  double *elec_w;
  int flat3;  // n3 = 1 with periodic X3: fluxes on the single k layer, copied
  // sides that continue into a neighbouring block of a decomposed grid (1)
  // rather than ending at a physical boundary (0): the fixup may average
  // over the first ghost layer there, which holds the neighbour's zones
  int xlo[3], xhi[3];
  // gamma, gamma - 1 and gamma (gamma - 1) split into float words (high, low)
  // for the float-float flux stage
  float gam_ff[2], gm1_ff[2], ggm1_ff[2], igam_ff[2], gf_ff[2];  // gf = (gamma - 1)/gamma
  const float *geomff, *connff;  // float-float mode: split geometry and connection
  int bc[3][2];
  const double *geom;
  const double *conn;
  const double *floors;
  Clock *clk;
};

// the inversion's and the bounds' adiabatic-index constants (IEEE host
// arithmetic: the values a per-zone division would give)
inline void set_gas_constants(StepArgs &A) {
  A.gk.gam = A.gam;
  A.gk.igam = A.igam;
  A.gk.gf = (A.gam - 1.0) / A.gam;
  A.gk.ubd = 2.0 * (A.gam - 1.0);
  A.gk.ubd_rcp = 1.0 / A.gk.ubd;
}

// the float-float words of the adiabatic-index constants
inline void set_ff_constants(StepArgs &A) {
  const double v[5] = {A.gam, A.gam - 1.0, A.gam * (A.gam - 1.0), A.igam, (A.gam - 1.0) / A.gam};
  float *o[5] = {A.gam_ff, A.gm1_ff, A.ggm1_ff, A.igam_ff, A.gf_ff};
  for (int q = 0; q < 5; q++) {
    o[q][0] = (float)v[q];
    o[q][1] = (float)(v[q] - (double)o[q][0]);
  }
}

void launch_geometry(const GeomArgs &A, cudaStream_t st);

// Single-grid kernels of the allocation-free flux entry point:
// zero clk->ctop_bits before a flux pass
void launch_ctop_reset(const StepArgs &A, cudaStream_t st);
// fluxes of P (fused reconstruction + LLF), with the interior ctop maxima
// into clk->ctop_bits
void launch_fluxes(const StepArgs &A, const double *P, double *F[3], cudaStream_t st);
// boundary flux fixes + flux-CT (emf scratch: 3 x ntot)
void launch_fix_ct(const StepArgs &A, double *F[3], double *emf, cudaStream_t st);

// FP32 copy of n doubles (clamped to the float range)
void launch_to_f32(long long n, const double *src, float *dst, cudaStream_t st);
// float-float split of n doubles: dst[0..n) high words, dst[n..2n) low words
void launch_to_ff(long long n, const double *src, float *dst, cudaStream_t st);
// max |corner divergence of sqrt(-g) B| and max |sqrt(-g) B^d| over the
// corners' zones, as double bit patterns into out[2] (device)
void launch_divb(const StepArgs &A, const double *P, unsigned long long *out, cudaStream_t st);
// pack interior <-> ghost layout
// nvar variables of ntot (interior <-> with ghosts)
void launch_pack(const Dims &D, const double *src, double *dst, int to_ghost, cudaStream_t st,
                 int nvar = NV);

}  // namespace grmhd
