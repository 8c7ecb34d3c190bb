// sim_impl.h -- host-side state of one simulation (the opaque grmhd_sim of
// include/grmhd.h), shared by the translation units that enqueue its work.
#pragma once

#include <utility>
#include <vector>

#include "../../include/grmhd.h"
#include "grmhd_impl.h"
#include "plan.h"

struct grmhd_sim {
  grmhd::Dims D;
  grmhd_grid grid;
  grmhd_metric metric;
  grmhd_params params;
  cudaStream_t st;
  double *P, *Ph, *F[3], *emf, *Lf, *Rf, *Uc;
  double *geom, *conn, *floors;
  float *Pf, *geomf;    // FP32 copies (mixed precision only)
  float *Pff, *geomff, *connff;  // split float-float copies (float-float mode only)
  // electrons only: entropies of the stage arrays, their fluxes, U_rho(P^n),
  // the faces' signal speeds
  double *K, *Kh, *FK[3], *Uek, *elec_w, *KLf, *KRf;
  int *pflag, *fflag;
  grmhd::Clock *clk;
  unsigned long long unrec_seen, dterr_seen;
  grmhd::StepArgs A;
  grmhd::Plan plan;  // the one-grid launch plan of the step
  // profiling: event pairs per class, launches per class
  int prof_on;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> *prof_ev;
  std::vector<cudaEvent_t> *ev_pool;
  long long launches[GRMHD_NKCLASS];
  double prof_ms[GRMHD_NKCLASS];
  // grmhd_step's CUDA graph of one cycle (replayed on gst, ordered after and
  // before st by gev), with the kernels it launches per class
  cudaStream_t gst;
  cudaEvent_t gev;
  cudaGraph_t graph;
  cudaGraphExec_t gexec;
  long long graph_launches[GRMHD_NKCLASS];
};

// drop grmhd_step's graph (the launch shapes it holds changed)
void sim_drop_graph(grmhd_sim *s);


// A block of a decomposed grid: the global index of its first interior
// zone, its size, and the sides that continue into a neighbouring block.
struct BlockSpec {
  int off[3], n[3], xlo[3], xhi[3];
};

// grmhd_create for a whole grid (blk == NULL) or for one block of a
// decomposed grid (grid: the global grid; params->bc with GRMHD_BC_EXCHANGE
// on the sides shared with other blocks; no validation: the caller
// validated the global problem).
int sim_create(const grmhd_grid *grid, const grmhd_metric *metric, const grmhd_params *params,
               void *stream, const BlockSpec *blk, grmhd_sim **out);
// the argument checks of grmhd_create
int validate_problem(const grmhd_grid *grid, const grmhd_metric *metric, const grmhd_params *params,
                     grmhd::Dims *Dout);
