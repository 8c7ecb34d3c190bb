// batch.cu -- the C ABI of batches: many independent grids advanced by one
// set of launches per step.
//
// A batch is a launch plan (plan.h) over its member simulations' buffers:
// each grid keeps its own buffers, geometry, boundary conditions,
// reconstruction, precision and device clock (so its own CFL time step and
// t_final), and the plan kernels are the ones a simulation stepped alone
// runs, so a grid's results are bitwise those of the same grid alone.  One
// step is the same number of launches whatever the number of grids;
// grmhd_batch_step can capture them once into a CUDA graph and replay it.
#include <cstring>
#include <new>
#include <set>
#include <vector>

#include "../../include/grmhd.h"
#include "grmhd_impl.h"
#include "plan.h"
#include "sim_impl.h"

using namespace grmhd;

struct grmhd_batch {
  int ngrid;
  std::vector<grmhd_sim *> sims;
  std::vector<cudaStream_t> member_streams;  // distinct streams of the members
  cudaStream_t st;                           // the batch's own stream
  cudaEvent_t ev;
  Plan plan;
  int launches_per_step;
  long long launches;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
};

static void batch_free(grmhd_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  plan_free(b->plan);
  if (b->ev) cudaEventDestroy(b->ev);
  if (b->st) cudaStreamDestroy(b->st);
}

extern "C" int grmhd_batch_create(grmhd_sim *const *sims, int nsims, grmhd_batch **out) {
  if (!sims || !out || nsims < 1) return GRMHD_ERR_INVALID;
  *out = nullptr;
  std::set<grmhd_sim *> seen;
  for (int g = 0; g < nsims; g++)
    if (!sims[g] || !seen.insert(sims[g]).second) return GRMHD_ERR_INVALID;  // null or repeated
  grmhd_batch *b = new (std::nothrow) grmhd_batch();
  if (!b) return GRMHD_ERR_NOMEM;
  b->ngrid = nsims;
  b->sims.assign(sims, sims + nsims);
  std::vector<StageItem> items(nsims);
  for (int g = 0; g < nsims; g++) {
    // the member's own one-grid plan item, read back from the device
    if (cudaMemcpy(&items[g], sims[g]->plan.items, sizeof(StageItem), cudaMemcpyDeviceToHost) !=
        cudaSuccess) {
      delete b;
      return GRMHD_ERR_CUDA;
    }
    bool dup = false;
    for (cudaStream_t q : b->member_streams) dup = dup || (q == sims[g]->st);
    if (!dup) b->member_streams.push_back(sims[g]->st);
  }
  int rc = plan_build(b->plan, items.data(), nsims);
  if (rc != GRMHD_OK) {
    delete b;
    return rc;
  }
  if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    batch_free(b);
    delete b;
    return GRMHD_ERR_CUDA;
  }
  *out = b;
  return GRMHD_OK;
}

extern "C" int grmhd_batch_destroy(grmhd_batch *b) {
  if (!b) return GRMHD_OK;
  if (b->st) cudaStreamSynchronize(b->st);
  batch_free(b);
  delete b;
  return GRMHD_OK;
}

extern "C" int grmhd_batch_step(grmhd_batch *b, int nsteps, int use_graph) {
  if (!b || nsteps < 0) return GRMHD_ERR_INVALID;
  if (nsteps == 0) return GRMHD_OK;
  // the batch's work follows everything already enqueued for its grids
  for (cudaStream_t q : b->member_streams) {
    if (cudaEventRecord(b->ev, q) != cudaSuccess) return GRMHD_ERR_CUDA;
    if (cudaStreamWaitEvent(b->st, b->ev, 0) != cudaSuccess) return GRMHD_ERR_CUDA;
  }
  if (use_graph && !b->exec) {
    if (cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return GRMHD_ERR_CUDA;
    const int nl = plan_steps(b->plan, 1, b->st, nullptr);
    cudaGraph_t gph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->st, &gph);
    if (e != cudaSuccess || !gph) {
      if (gph) cudaGraphDestroy(gph);
      cudaGetLastError();
      return GRMHD_ERR_CUDA;
    }
    if (cudaGraphInstantiate(&b->exec, gph, 0) != cudaSuccess) {
      cudaGraphDestroy(gph);
      b->exec = nullptr;
      cudaGetLastError();
      return GRMHD_ERR_CUDA;
    }
    b->graph = gph;
    b->launches_per_step = nl;
  }
  for (int n = 0; n < nsteps; n++) {
    if (use_graph) {
      if (cudaGraphLaunch(b->exec, b->st) != cudaSuccess) return GRMHD_ERR_CUDA;
      b->launches += b->launches_per_step;
    } else {
      b->launches_per_step = plan_steps(b->plan, 1, b->st, nullptr);
      b->launches += b->launches_per_step;
    }
  }
  if (cudaGetLastError() != cudaSuccess) return GRMHD_ERR_CUDA;
  // and everything enqueued for a grid later follows the batch's work
  if (cudaEventRecord(b->ev, b->st) != cudaSuccess) return GRMHD_ERR_CUDA;
  for (cudaStream_t q : b->member_streams)
    if (cudaStreamWaitEvent(q, b->ev, 0) != cudaSuccess) return GRMHD_ERR_CUDA;
  return GRMHD_OK;
}

static void drop_graph(grmhd_batch *b) {
  if (b->exec) {  // the graph holds the old launch shapes
    cudaGraphExecDestroy(b->exec);
    cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
  }
}

extern "C" int grmhd_batch_set_launch(grmhd_batch *b, int kclass, int threads, int order) {
  if (!b) return GRMHD_ERR_INVALID;
  static const int recon[] = {PC_RECON0, PC_RECON1, PC_RECON2, PC_TOF32, PC_RECON01X, PC_RECON2X};
  static const int flux[] = {PC_FACE0,  PC_FACE1,  PC_FACE2,  PC_FACE0E, PC_FACE1E, PC_FACE2E,
                             PC_FACE0F, PC_FACE1F, PC_FACE2F, PC_FACE0X, PC_FACE1X, PC_FACE2X};
  static const int zone[] = {PC_ZONE, PC_UPD64, PC_UPDX};
  const int *cls = nullptr;
  int ncls = 0;
  if (kclass == GRMHD_K_RECON) {
    cls = recon;
    ncls = 6;
  } else if (kclass == GRMHD_K_FLUX) {
    cls = flux;
    ncls = 12;
  } else if (kclass == GRMHD_K_UPDATE) {
    cls = zone;
    ncls = 3;
  } else {
    return GRMHD_ERR_INVALID;
  }
  if (threads < 64 || threads > 256 || threads % 32 || order < 0 || order >= PLAN_SCHED_N)
    return GRMHD_ERR_INVALID;
  drop_graph(b);
  for (int q = 0; q < ncls; q++) {
    const int rc = plan_set_class(b->plan, cls[q], threads, order);
    if (rc != GRMHD_OK) return rc;
  }
  return GRMHD_OK;
}

extern "C" int grmhd_batch_autotune(grmhd_batch *b, int trials, double *ms_before,
                                    double *ms_after) {
  if (!b || trials < 1) return GRMHD_ERR_INVALID;
  // the members' pending work first (the trials read their current state)
  for (cudaStream_t q : b->member_streams)
    if (cudaStreamSynchronize(q) != cudaSuccess) return GRMHD_ERR_CUDA;
  const int rc = plan_autotune(b->plan, trials, b->st, ms_before, ms_after);
  drop_graph(b);
  return rc;
}

extern "C" int grmhd_batch_get_info(grmhd_batch *b, grmhd_batch_info *out) {
  if (!b || !out) return GRMHD_ERR_INVALID;
  out->ngrid = b->ngrid;
  out->zones = b->plan.zones;
  out->launches_per_step = b->launches_per_step;
  out->launches = b->launches;
  out->graph = b->exec ? 1 : 0;
  out->tuned = b->plan.tuned;
  out->recon_walk = b->plan.ngrid > 0 ? b->plan.host_items[0].A.rwalk : 0;
  return GRMHD_OK;
}

extern "C" int grmhd_batch_sync(grmhd_batch *b) {
  if (!b) return GRMHD_ERR_INVALID;
  return cudaStreamSynchronize(b->st) == cudaSuccess ? GRMHD_OK : GRMHD_ERR_CUDA;
}
