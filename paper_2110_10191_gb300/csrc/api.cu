// api.cu -- the C ABI (include/grmhd.h): simulation lifetime, state I/O and
// the host-side driver that enqueues the kernels of each step on the
// simulation's stream.  The step needs no host round trip: the CFL time
// step, the clock and the statistics live in device memory.
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/grmhd.h"
#include "grmhd_dev.cuh"
#include "grmhd_impl.h"
#include "plan.h"
#include "sim_impl.h"

using namespace grmhd;


// Counts the launches of each kernel class and, when profiling, records an
// event pair on the stream around each launch.
// Counts the launches per class of a captured cycle.
struct CountHook : PlanHook {
  long long *n;
  explicit CountHook(long long *n_) : n(n_) {}
  void begin(int cls, int nlaunch) override { n[cls] += nlaunch; }
  void end(int) override {}
};

struct SimHook : PlanHook {
  grmhd_sim *s;
  cudaEvent_t e0;
  explicit SimHook(grmhd_sim *s_) : s(s_), e0(nullptr) {}
  void begin(int cls, int nlaunch) override {
    s->launches[cls] += nlaunch;
    if (s->prof_on) {
      e0 = take_event();
      cudaEventRecord(e0, s->st);
    }
  }
  void end(int cls) override {
    if (s->prof_on) {
      cudaEvent_t e1 = take_event();
      cudaEventRecord(e1, s->st);
      s->prof_ev->push_back({cls, {e0, e1}});
    }
  }
  cudaEvent_t take_event() {
    if (!s->ev_pool->empty()) {
      cudaEvent_t e = s->ev_pool->back();
      s->ev_pool->pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
};

#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) return GRMHD_ERR_CUDA; \
  } while (0)

static int launched(void) { return (cudaGetLastError() == cudaSuccess) ? GRMHD_OK : GRMHD_ERR_CUDA; }

static void collect_profile(grmhd_sim *s) {
  if (!s->prof_ev) return;
  for (auto &p : *s->prof_ev) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, p.second.first, p.second.second) == cudaSuccess)
      s->prof_ms[p.first] += ms;
    s->ev_pool->push_back(p.second.first);
    s->ev_pool->push_back(p.second.second);
  }
  s->prof_ev->clear();
}

static void free_all(grmhd_sim *s) {
  if (s->prof_ev) {
    cudaStreamSynchronize(s->st);
    collect_profile(s);
    for (cudaEvent_t e : *s->ev_pool) cudaEventDestroy(e);
    delete s->prof_ev;
    delete s->ev_pool;
    s->prof_ev = nullptr;
    s->ev_pool = nullptr;
  }
  sim_drop_graph(s);
  if (s->gev) cudaEventDestroy(s->gev);
  if (s->gst) cudaStreamDestroy(s->gst);
  s->gev = nullptr;
  s->gst = nullptr;
  plan_free(s->plan);
  double *d[] = {s->P,      s->Ph,    s->F[0], s->F[1], s->F[2],  s->emf,
                 s->Lf,     s->Rf,    s->Uc,   s->geom, s->conn,  s->floors,
                 s->K,      s->Kh,    s->FK[0], s->FK[1], s->FK[2], s->Uek,
                 s->elec_w, s->KLf, s->KRf};
  for (double *p : d)
    if (p) cudaFree(p);
  if (s->Pf) cudaFree(s->Pf);
  if (s->geomf) cudaFree(s->geomf);
  if (s->Pff) cudaFree(s->Pff);
  if (s->geomff) cudaFree(s->geomff);
  if (s->connff) cudaFree(s->connff);
  if (s->pflag) cudaFree(s->pflag);
  if (s->fflag) cudaFree(s->fflag);
  if (s->clk) cudaFree(s->clk);
}

// Arguments of grmhd_create: GRMHD_OK and the dimensions, or GRMHD_ERR_INVALID.
int validate_problem(const grmhd_grid *grid, const grmhd_metric *metric, const grmhd_params *params,
                     Dims *Dout) {
  if (!grid || !metric || !params) return GRMHD_ERR_INVALID;
  const int n[3] = {grid->n1, grid->n2, grid->n3};
  const double xmin[3] = {grid->x1min, grid->x2min, grid->x3min};
  const double xmax[3] = {grid->x1max, grid->x2max, grid->x3max};
  long long tot = 1;
  Dims D;
  for (int d = 0; d < 3; d++) {
    if (n[d] < 1 || n[d] > (1 << 20)) return GRMHD_ERR_INVALID;
    if (!(xmax[d] > xmin[d])) return GRMHD_ERR_INVALID;
    D.n[d] = n[d];
    D.s[d] = n[d] + 2 * NG;
    tot *= (long long)(n[d] + 2 * NG);
  }
  if (tot >= (1ll << 31)) return GRMHD_ERR_INVALID;
  D.ntot = tot;
  D.n2d = (long long)D.s[0] * D.s[1];
  if (metric->kind != GRMHD_METRIC_MINKOWSKI && metric->kind != GRMHD_METRIC_MKS_KERR)
    return GRMHD_ERR_INVALID;
  if (metric->kind == GRMHD_METRIC_MKS_KERR && !(fabs(metric->a) < 1.0)) return GRMHD_ERR_INVALID;
  if (!(params->gamma > 1.0) || !(params->cfl > 0.0)) return GRMHD_ERR_INVALID;
  if (params->recon != GRMHD_RECON_MC && params->recon != GRMHD_RECON_WENO5) return GRMHD_ERR_INVALID;
  if (params->precision != GRMHD_PREC_FP64 && params->precision != GRMHD_PREC_MIXED &&
      params->precision != GRMHD_PREC_FF && params->precision != GRMHD_PREC_MIXED_FF)
    return GRMHD_ERR_INVALID;
  if (params->floors_on && metric->kind != GRMHD_METRIC_MKS_KERR) return GRMHD_ERR_INVALID;
  if (params->floor_frame != GRMHD_FLOOR_FLUID && params->floor_frame != GRMHD_FLOOR_DRIFT)
    return GRMHD_ERR_INVALID;
  const grmhd_electrons &e = params->electrons;
  if (e.model < GRMHD_ELEC_OFF || e.model > GRMHD_ELEC_HOWES) return GRMHD_ERR_INVALID;
  if (e.model != GRMHD_ELEC_OFF) {
    if (!(e.game > 1.0) || !(e.gamp > 1.0)) return GRMHD_ERR_INVALID;
    if (!(e.tpte_min >= 0.0) || !(e.tpte_max >= e.tpte_min)) return GRMHD_ERR_INVALID;
    if (e.model == GRMHD_ELEC_CONSTANT && !(e.fel >= 0.0 && e.fel <= 1.0)) return GRMHD_ERR_INVALID;
  }
  for (int d = 0; d < 3; d++)
    for (int sd = 0; sd < 2; sd++) {
      const int b = params->bc[d][sd];
      if (b < 0 || b > 3) return GRMHD_ERR_INVALID;
      if (b == GRMHD_BC_OUTFLOW && d != 0) return GRMHD_ERR_INVALID;
      if (b == GRMHD_BC_POLAR && (d != 1 || n[1] < NG)) return GRMHD_ERR_INVALID;
      if ((b == GRMHD_BC_PERIODIC) != (params->bc[d][1 - sd] == GRMHD_BC_PERIODIC))
        return GRMHD_ERR_INVALID;
    }
  if (Dout) *Dout = D;
  return GRMHD_OK;
}

// (grids with electrons take the full extent: their entropy fluxes are not
// replicated)
static int flat3_of(const Dims &D, const grmhd_params *params) {
  return (D.n[2] == 1 && params->bc[2][0] == GRMHD_BC_PERIODIC && !params->electrons.model) ? 1 : 0;
}

extern "C" int grmhd_footprint(const grmhd_grid *grid, const grmhd_metric *metric,
                               const grmhd_params *params, size_t *bytes) {
  Dims D;
  if (!bytes) return GRMHD_ERR_INVALID;
  const int rc = validate_problem(grid, metric, params, &D);
  if (rc != GRMHD_OK) return rc;
  const size_t tot = (size_t)D.ntot, n2d = (size_t)D.n2d;
  size_t b = sizeof(double) * NV * tot * 8                 // P, Ph, F1..3, Lf, Rf, Uc
             + sizeof(double) * 3 * tot                    // EMFs
             + sizeof(double) * (NLOC * G_NCOMP + C_NCOMP + 2) * n2d  // geometry, connection, bounds
             + sizeof(int) * 2 * tot + sizeof(Clock);     // flags, clock
  const int pr = params->precision;
  if (pr == GRMHD_PREC_MIXED || pr == GRMHD_PREC_MIXED_FF)  // FP32 stage input and geometry
    b += sizeof(float) * NV * tot + sizeof(float) * NLOC * G_NCOMP * n2d;
  if (pr == GRMHD_PREC_FF)  // split stage input
    b += 2 * sizeof(float) * NV * tot;
  if (pr == GRMHD_PREC_FF || pr == GRMHD_PREC_MIXED_FF)  // split geometry and connection
    b += 2 * sizeof(float) * (NLOC * G_NCOMP + C_NCOMP) * n2d;
  if (params->electrons.model)  // K, Kh, FK[3], KLf, KRf (2 each), Uek, elec_w (6)
    b += sizeof(double) * 21 * tot;
  b += (size_t)plan_bytes(D, flat3_of(D, params), params->precision,
                         params->floors_on && params->floor_frame == GRMHD_FLOOR_DRIFT,
                         params->electrons.model != GRMHD_ELEC_OFF);
  *bytes = b;
  return GRMHD_OK;
}

int sim_create(const grmhd_grid *grid, const grmhd_metric *metric, const grmhd_params *params,
               void *stream, const BlockSpec *blk, grmhd_sim **out) {
  if (!out) return GRMHD_ERR_INVALID;
  *out = nullptr;
  if (!blk) {
    const int rc = validate_problem(grid, metric, params, nullptr);
    if (rc != GRMHD_OK) return rc;
  }
  // a block: its own size, the global grid's coordinates
  const int gn[3] = {grid->n1, grid->n2, grid->n3};
  const int n[3] = {blk ? blk->n[0] : gn[0], blk ? blk->n[1] : gn[1], blk ? blk->n[2] : gn[2]};
  const double xmin[3] = {grid->x1min, grid->x2min, grid->x3min};
  const double xmax[3] = {grid->x1max, grid->x2max, grid->x3max};
  long long tot = 1;
  for (int d = 0; d < 3; d++) tot *= (long long)(n[d] + 2 * NG);

  grmhd_sim *s = new (std::nothrow) grmhd_sim();
  if (!s) return GRMHD_ERR_NOMEM;
  memset((void *)s, 0, sizeof(*s));
  s->prof_ev = new (std::nothrow) std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>>();
  s->ev_pool = new (std::nothrow) std::vector<cudaEvent_t>();
  if (!s->prof_ev || !s->ev_pool) {
    delete s->prof_ev;
    delete s->ev_pool;
    delete s;
    return GRMHD_ERR_NOMEM;
  }
  s->grid = *grid;
  s->metric = *metric;
  s->params = *params;
  s->st = (cudaStream_t)stream;
  Dims &D = s->D;
  for (int d = 0; d < 3; d++) {
    D.n[d] = n[d];
    D.s[d] = n[d] + 2 * NG;
  }
  D.ntot = tot;
  D.n2d = (long long)D.s[0] * D.s[1];
  const size_t fb = sizeof(double) * NV * (size_t)tot;
  bool ok = cudaMalloc(&s->P, fb) == cudaSuccess && cudaMalloc(&s->Ph, fb) == cudaSuccess &&
            cudaMalloc(&s->F[0], fb) == cudaSuccess && cudaMalloc(&s->F[1], fb) == cudaSuccess &&
            cudaMalloc(&s->F[2], fb) == cudaSuccess && cudaMalloc(&s->Lf, fb) == cudaSuccess &&
            cudaMalloc(&s->Rf, fb) == cudaSuccess && cudaMalloc(&s->Uc, fb) == cudaSuccess &&
            cudaMalloc(&s->emf, sizeof(double) * 3 * (size_t)tot) == cudaSuccess &&
            cudaMalloc(&s->geom, sizeof(double) * NLOC * G_NCOMP * (size_t)D.n2d) == cudaSuccess &&
            cudaMalloc(&s->conn, sizeof(double) * C_NCOMP * (size_t)D.n2d) == cudaSuccess &&
            cudaMalloc(&s->floors, sizeof(double) * 2 * (size_t)D.n2d) == cudaSuccess &&
            cudaMalloc(&s->pflag, sizeof(int) * (size_t)tot) == cudaSuccess &&
            cudaMalloc(&s->fflag, sizeof(int) * (size_t)tot) == cudaSuccess &&
            cudaMalloc(&s->clk, sizeof(Clock)) == cudaSuccess;
  const int prec = params->precision;
  if (ok && (prec == GRMHD_PREC_MIXED || prec == GRMHD_PREC_MIXED_FF))
    ok = cudaMalloc(&s->Pf, sizeof(float) * NV * (size_t)tot) == cudaSuccess &&
         cudaMalloc(&s->geomf, sizeof(float) * NLOC * G_NCOMP * (size_t)D.n2d) == cudaSuccess;
  if (ok && prec == GRMHD_PREC_FF)
    ok = cudaMalloc(&s->Pff, 2 * sizeof(float) * NV * (size_t)tot) == cudaSuccess;
  if (ok && (prec == GRMHD_PREC_FF || prec == GRMHD_PREC_MIXED_FF))
    ok = cudaMalloc(&s->geomff, 2 * sizeof(float) * NLOC * G_NCOMP * (size_t)D.n2d) == cudaSuccess &&
         cudaMalloc(&s->connff, 2 * sizeof(float) * C_NCOMP * (size_t)D.n2d) == cudaSuccess;
  const bool elec = params->electrons.model != GRMHD_ELEC_OFF;
  const size_t kb = sizeof(double) * 2 * (size_t)tot;
  if (ok && elec)
    ok = cudaMalloc(&s->K, kb) == cudaSuccess && cudaMalloc(&s->Kh, kb) == cudaSuccess &&
         cudaMalloc(&s->FK[0], kb) == cudaSuccess && cudaMalloc(&s->FK[1], kb) == cudaSuccess &&
         cudaMalloc(&s->FK[2], kb) == cudaSuccess && cudaMalloc(&s->KLf, kb) == cudaSuccess &&
         cudaMalloc(&s->KRf, kb) == cudaSuccess &&
         cudaMalloc(&s->Uek, sizeof(double) * (size_t)tot) == cudaSuccess &&
         cudaMalloc(&s->elec_w, sizeof(double) * 6 * (size_t)tot) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_all(s);
    delete s;
    return GRMHD_ERR_NOMEM;
  }
  int rc = GRMHD_OK;
  cudaStream_t st = s->st;
  if (elec)
    for (double *q : {s->K, s->Kh, s->FK[0], s->FK[1], s->FK[2], s->KLf, s->KRf})
      if (cudaMemsetAsync(q, 0, kb, st) != cudaSuccess) rc = GRMHD_ERR_CUDA;
  // zero every field so that entries outside the computed ranges read as 0
  if (cudaMemsetAsync(s->P, 0, fb, st) != cudaSuccess || cudaMemsetAsync(s->Ph, 0, fb, st) != cudaSuccess ||
      cudaMemsetAsync(s->F[0], 0, fb, st) != cudaSuccess || cudaMemsetAsync(s->F[1], 0, fb, st) != cudaSuccess ||
      cudaMemsetAsync(s->F[2], 0, fb, st) != cudaSuccess ||
      cudaMemsetAsync(s->emf, 0, sizeof(double) * 3 * (size_t)tot, st) != cudaSuccess ||
      cudaMemsetAsync(s->pflag, 0, sizeof(int) * (size_t)tot, st) != cudaSuccess ||
      cudaMemsetAsync(s->fflag, 0, sizeof(int) * (size_t)tot, st) != cudaSuccess)
    rc = GRMHD_ERR_CUDA;
  Clock c0;
  memset(&c0, 0, sizeof(c0));
  c0.t_final = params->t_final;
  if (rc == GRMHD_OK && cudaMemcpyAsync(s->clk, &c0, sizeof(c0), cudaMemcpyHostToDevice, st) != cudaSuccess)
    rc = GRMHD_ERR_CUDA;
  GeomArgs G;
  G.D = D;
  G.kind = metric->kind;
  G.a = metric->a;
  G.h = metric->hslope;
  G.gam = params->gamma;
  for (int d = 0; d < 3; d++) {
    G.xmin[d] = xmin[d];
    G.dx[d] = (xmax[d] - xmin[d]) / gn[d];
    G.off[d] = blk ? blk->off[d] : 0;
  }
  G.geom = s->geom;
  G.conn = s->conn;
  G.floors = s->floors;
  if (rc == GRMHD_OK) {
    launch_geometry(G, st);
    if (s->geomf) launch_to_f32((long long)NLOC * G_NCOMP * D.n2d, s->geom, s->geomf, st);
    if (s->geomff) launch_to_ff((long long)NLOC * G_NCOMP * D.n2d, s->geom, s->geomff, st);
    if (s->connff) launch_to_ff((long long)C_NCOMP * D.n2d, s->conn, s->connff, st);
    rc = launched();
  }
  if (rc == GRMHD_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = GRMHD_ERR_CUDA;
  if (rc != GRMHD_OK) {
    free_all(s);
    delete s;
    return rc;
  }
  StepArgs &A = s->A;
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
  A.floor_drift = params->floors_on && params->floor_frame == GRMHD_FLOOR_DRIFT;
  A.elec = params->electrons.model;
  A.game = params->electrons.game;
  A.gamp = params->electrons.gamp;
  A.fel_const = params->electrons.fel;
  A.tpte_min = params->electrons.tpte_min;
  A.tpte_max = params->electrons.tpte_max;
  A.elec_w = s->elec_w;
  for (int d = 0; d < 3; d++)
    for (int sd = 0; sd < 2; sd++) A.bc[d][sd] = params->bc[d][sd];
  A.flat3 = flat3_of(D, params);
  for (int d = 0; d < 3; d++) {
    A.xlo[d] = blk ? blk->xlo[d] : 0;
    A.xhi[d] = blk ? blk->xhi[d] : 0;
  }
  set_ff_constants(A);
  set_gas_constants(A);
  A.geomff = s->geomff;
  A.connff = s->connff;
  A.geom = s->geom;
  A.conn = s->conn;
  A.floors = s->floors;
  A.clk = s->clk;
  StageItem it;
  memset(&it, 0, sizeof(it));
  it.A = A;
  it.P = s->P;
  it.Ph = s->Ph;
  for (int d = 0; d < 3; d++) it.F[d] = s->F[d];
  it.emf = s->emf;
  it.Lf = s->Lf;
  it.Rf = s->Rf;
  it.Uc = s->Uc;
  it.pflag = s->pflag;
  it.fflag = s->fflag;
  it.Pf = s->Pf;
  it.geomf = s->geomf;
  it.Pff = s->Pff;
  it.geomff = s->geomff;
  it.prec = params->precision;
  it.K = s->K;
  it.Kh = s->Kh;
  for (int d = 0; d < 3; d++) it.FK[d] = s->FK[d];
  it.Uek = s->Uek;
  it.KLf = s->KLf;
  it.KRf = s->KRf;
  rc = plan_build(s->plan, &it, 1);
  if (rc != GRMHD_OK) {
    free_all(s);
    delete s;
    return rc;
  }
  *out = s;
  return GRMHD_OK;
}

extern "C" int grmhd_create(const grmhd_grid *grid, const grmhd_metric *metric,
                            const grmhd_params *params, void *stream, grmhd_sim **out) {
  return sim_create(grid, metric, params, stream, nullptr, out);
}

extern "C" int grmhd_destroy(grmhd_sim *s) {
  if (!s) return GRMHD_OK;
  cudaStreamSynchronize(s->st);
  free_all(s);
  delete s;
  return GRMHD_OK;
}

static int set_common(grmhd_sim *s, const double *P, int on_device, int ghost) {
  if (!s || !P) return GRMHD_ERR_INVALID;
  const Dims &D = s->D;
  const long long nz = (long long)D.n[0] * D.n[1] * D.n[2];
  const size_t bytes = sizeof(double) * NV * (size_t)(ghost ? D.ntot : nz);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (ghost) {
    CK(cudaMemcpyAsync(s->P, P, bytes, kind, s->st));
  } else {
    CK(cudaMemcpyAsync(s->Ph, P, bytes, kind, s->st));  // Ph is scratch between steps
    launch_pack(D, s->Ph, s->P, 1, s->st);
  }
  {
    SimHook h(s);
    plan_bounds(s->plan, 0, s->st, &h);
  }
  // the ghosts of a fixed side keep their set values in both stage arrays
  CK(cudaMemcpyAsync(s->Ph, s->P, sizeof(double) * NV * (size_t)D.ntot, cudaMemcpyDeviceToDevice,
                     s->st));
  if (s->K)
    CK(cudaMemcpyAsync(s->Kh, s->K, sizeof(double) * 2 * (size_t)D.ntot, cudaMemcpyDeviceToDevice,
                       s->st));
  int rc = launched();
  if (rc != GRMHD_OK) return rc;
  if (!on_device) CK(cudaStreamSynchronize(s->st));
  return GRMHD_OK;
}

extern "C" int grmhd_set_prims(grmhd_sim *s, const double *P, int on_device) {
  return set_common(s, P, on_device, 0);
}

extern "C" int grmhd_set_prims_ghost(grmhd_sim *s, const double *P, int on_device) {
  return set_common(s, P, on_device, 1);
}

extern "C" int grmhd_set_electrons(grmhd_sim *s, const double *K, int with_ghosts, int on_device) {
  if (!s || !K || !s->K) return GRMHD_ERR_INVALID;
  const Dims &D = s->D;
  const long long nz = (long long)D.n[0] * D.n[1] * D.n[2];
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (with_ghosts) {
    CK(cudaMemcpyAsync(s->K, K, sizeof(double) * 2 * (size_t)D.ntot, kind, s->st));
  } else {
    CK(cudaMemcpyAsync(s->Kh, K, sizeof(double) * 2 * (size_t)nz, kind, s->st));  // scratch
    launch_pack(D, s->Kh, s->K, 1, s->st, 2);
  }
  {
    SimHook h(s);
    plan_bounds(s->plan, 0, s->st, &h);  // refills the primitives' ghosts too (unchanged)
  }
  CK(cudaMemcpyAsync(s->Kh, s->K, sizeof(double) * 2 * (size_t)D.ntot, cudaMemcpyDeviceToDevice,
                     s->st));
  CK(cudaMemcpyAsync(s->Ph, s->P, sizeof(double) * NV * (size_t)D.ntot, cudaMemcpyDeviceToDevice,
                     s->st));
  int rc = launched();
  if (rc != GRMHD_OK) return rc;
  if (!on_device) CK(cudaStreamSynchronize(s->st));
  return GRMHD_OK;
}

extern "C" int grmhd_get_electrons(grmhd_sim *s, double *K, int with_ghosts, int on_device) {
  if (!s || !K || !s->K) return GRMHD_ERR_INVALID;
  const Dims &D = s->D;
  const long long nz = (long long)D.n[0] * D.n[1] * D.n[2];
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (with_ghosts) {
    CK(cudaMemcpyAsync(K, s->K, sizeof(double) * 2 * (size_t)D.ntot, kind, s->st));
  } else {
    launch_pack(D, s->K, s->Kh, 0, s->st, 2);
    int rc = launched();
    if (rc != GRMHD_OK) return rc;
    CK(cudaMemcpyAsync(K, s->Kh, sizeof(double) * 2 * (size_t)nz, kind, s->st));
  }
  if (!on_device) CK(cudaStreamSynchronize(s->st));
  return GRMHD_OK;
}

extern "C" int grmhd_get_prims(grmhd_sim *s, double *P, int with_ghosts, int on_device) {
  if (!s || !P) return GRMHD_ERR_INVALID;
  const Dims &D = s->D;
  const long long nz = (long long)D.n[0] * D.n[1] * D.n[2];
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (with_ghosts) {
    CK(cudaMemcpyAsync(P, s->P, sizeof(double) * NV * (size_t)D.ntot, kind, s->st));
  } else {
    launch_pack(D, s->P, s->Ph, 0, s->st);
    int rc = launched();
    if (rc != GRMHD_OK) return rc;
    CK(cudaMemcpyAsync(P, s->Ph, sizeof(double) * NV * (size_t)nz, kind, s->st));
  }
  if (!on_device) CK(cudaStreamSynchronize(s->st));
  return GRMHD_OK;
}

static int read_stats(grmhd_sim *s, grmhd_stats *out, bool check) {
  Clock c;
  CK(cudaMemcpyAsync(&c, s->clk, sizeof(c), cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  if (out) {
    out->t = c.t;
    out->dt = c.dt;
    out->steps = c.steps;
    out->inv_failures = (long long)c.counters[0];
    out->floor_hits = (long long)c.counters[1];
    out->unrecoverable = (long long)c.counters[2];
  }
  int rc = GRMHD_OK;
  if (check && c.counters[2] > s->unrec_seen) rc = GRMHD_ERR_INVERSION;
  if (check && c.counters[3] > s->dterr_seen) rc = GRMHD_ERR_DT;
  s->unrec_seen = c.counters[2];
  s->dterr_seen = c.counters[3];
  return rc;
}

void sim_drop_graph(grmhd_sim *s) {
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  if (s->graph) cudaGraphDestroy(s->graph);
  s->gexec = nullptr;
  s->graph = nullptr;
}

// nsteps cycles as replays of a CUDA graph of one cycle, captured on first
// use on the simulation's own capture stream, which waits for the work
// already enqueued on st and which st then waits for.  The graph runs the
// same kernels with the same arguments as direct launches.
static int step_graph(grmhd_sim *s, int nsteps) {
  if (!s->gst) {
    if (cudaStreamCreateWithFlags(&s->gst, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->gev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return GRMHD_ERR_CUDA;
    }
  }
  CK(cudaEventRecord(s->gev, s->st));
  CK(cudaStreamWaitEvent(s->gst, s->gev, 0));
  if (!s->gexec) {
    long long n[GRMHD_NKCLASS] = {0};
    CK(cudaStreamBeginCapture(s->gst, cudaStreamCaptureModeThreadLocal));
    {
      CountHook h(n);
      plan_steps(s->plan, 1, s->gst, &h);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s->gst, &g);
    if (e != cudaSuccess || !g || cudaGraphInstantiate(&s->gexec, g, 0) != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      s->gexec = nullptr;
      cudaGetLastError();
      return GRMHD_ERR_CUDA;
    }
    s->graph = g;
    memcpy(s->graph_launches, n, sizeof(n));
  }
  for (int q = 0; q < nsteps; q++) CK(cudaGraphLaunch(s->gexec, s->gst));
  for (int c = 0; c < GRMHD_NKCLASS; c++) s->launches[c] += nsteps * s->graph_launches[c];
  CK(cudaEventRecord(s->gev, s->gst));
  CK(cudaStreamWaitEvent(s->st, s->gev, 0));
  return GRMHD_OK;
}

extern "C" int grmhd_step(grmhd_sim *s, int nsteps, grmhd_stats *stats) {
  if (!s || nsteps < 0) return GRMHD_ERR_INVALID;
  if (nsteps >= 2 && !s->prof_on) {  // many cycles, no per-class timing: replay a graph
    const int rc = step_graph(s, nsteps);
    if (rc != GRMHD_OK) return rc;
  } else {
    SimHook h(s);
    plan_steps(s->plan, nsteps, s->st, &h);
  }
  int rc = launched();
  if (rc != GRMHD_OK) return rc;
  if (stats) return read_stats(s, stats, true);
  return GRMHD_OK;
}

extern "C" int grmhd_get_stats(grmhd_sim *s, grmhd_stats *stats) {
  if (!s || !stats) return GRMHD_ERR_INVALID;
  return read_stats(s, stats, false);
}

extern "C" int grmhd_set_time(grmhd_sim *s, double t, double dt_prev, long long steps) {
  if (!s) return GRMHD_ERR_INVALID;
  Clock c;
  CK(cudaMemcpyAsync(&c, s->clk, sizeof(c), cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  c.t = t;
  c.dt = dt_prev;
  c.dt_prev = dt_prev;
  c.steps = steps;
  CK(cudaMemcpyAsync(s->clk, &c, sizeof(c), cudaMemcpyHostToDevice, s->st));
  CK(cudaStreamSynchronize(s->st));
  return GRMHD_OK;
}

extern "C" int grmhd_predictor(grmhd_sim *s) {
  if (!s) return GRMHD_ERR_INVALID;
  {
    SimHook h(s);
    plan_stage(s->plan, 0, 0, s->st, &h);
  }
  int rc = launched();
  if (rc != GRMHD_OK) return rc;
  // P <- P^{n+1/2} (ghosts included)
  CK(cudaMemcpyAsync(s->P, s->Ph, sizeof(double) * NV * (size_t)s->D.ntot, cudaMemcpyDeviceToDevice,
                     s->st));
  if (s->K)
    CK(cudaMemcpyAsync(s->K, s->Kh, sizeof(double) * 2 * (size_t)s->D.ntot,
                       cudaMemcpyDeviceToDevice, s->st));
  return read_stats(s, nullptr, true);
}

extern "C" int grmhd_get_fluxes(grmhd_sim *s, double *F, double *ctop) {
  if (!s || !F) return GRMHD_ERR_INVALID;
  {
    SimHook h(s);
    plan_fluxes(s->plan, 0, s->st, &h);
    plan_fix_ct(s->plan, s->st, &h);
  }
  int rc = launched();
  if (rc != GRMHD_OK) return rc;
  const size_t per = sizeof(double) * NV * (size_t)s->D.ntot;
  for (int d = 0; d < 3; d++)
    CK(cudaMemcpyAsync((char *)F + d * per, s->F[d], per, cudaMemcpyDeviceToHost, s->st));
  Clock c;
  CK(cudaMemcpyAsync(&c, s->clk, sizeof(c), cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  if (ctop) {
    for (int d = 0; d < 3; d++) {
      double v;
      memcpy(&v, &c.ctop_bits[d], sizeof(v));
      ctop[d] = v;
    }
  }
  return GRMHD_OK;
}

extern "C" int grmhd_next_dt(grmhd_sim *s, double *dt) {
  if (!s || !dt) return GRMHD_ERR_INVALID;
  Clock c0, c1;
  CK(cudaMemcpyAsync(&c0, s->clk, sizeof(c0), cudaMemcpyDeviceToHost, s->st));
  {
    SimHook h(s);
    plan_fluxes(s->plan, 0, s->st, &h);
    plan_clock(s->plan, 1, s->st, &h);
  }
  int rc = launched();
  if (rc != GRMHD_OK) return rc;
  CK(cudaMemcpyAsync(&c1, s->clk, sizeof(c1), cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  *dt = c1.dt;
  c1.dt = c0.dt;  // leave the reported last-step dt unchanged
  CK(cudaMemcpyAsync(s->clk, &c1, sizeof(c1), cudaMemcpyHostToDevice, s->st));
  CK(cudaStreamSynchronize(s->st));
  return GRMHD_OK;
}

extern "C" int grmhd_get_flags(grmhd_sim *s, int *pflag, int *fflag) {
  if (!s || !pflag || !fflag) return GRMHD_ERR_INVALID;
  const Dims &D = s->D;
  std::vector<int> a((size_t)D.ntot), b((size_t)D.ntot);
  CK(cudaMemcpyAsync(a.data(), s->pflag, sizeof(int) * a.size(), cudaMemcpyDeviceToHost, s->st));
  CK(cudaMemcpyAsync(b.data(), s->fflag, sizeof(int) * b.size(), cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  long long o = 0;
  for (int k = 0; k < D.n[2]; k++)
    for (int j = 0; j < D.n[1]; j++)
      for (int i = 0; i < D.n[0]; i++, o++) {
        const long long c = ((long long)(k + NG) * D.s[1] + (j + NG)) * D.s[0] + (i + NG);
        pflag[o] = a[(size_t)c];
        fflag[o] = b[(size_t)c];
      }
  return GRMHD_OK;
}

extern "C" int grmhd_get_geometry(grmhd_sim *s, int loc, double *out) {
  if (!s || !out || loc < 0 || loc > 3) return GRMHD_ERR_INVALID;
  const long long n2d = s->D.n2d;
  if (loc == 3) {
    std::vector<double> c((size_t)(C_NCOMP * n2d));
    CK(cudaMemcpyAsync(c.data(), s->conn, sizeof(double) * c.size(), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    for (int l = 0; l < 4; l++)
      for (int m = 0; m < 4; m++)
        for (int n = 0; n < 4; n++)
          memcpy(out + ((l * 4 + m) * 4 + n) * n2d, c.data() + (l * 10 + SY(m, n)) * n2d,
                 sizeof(double) * (size_t)n2d);
    return GRMHD_OK;
  }
  std::vector<double> g((size_t)(G_NCOMP * n2d));
  CK(cudaMemcpyAsync(g.data(), s->geom + (long long)loc * G_NCOMP * n2d, sizeof(double) * g.size(),
                     cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  for (int m = 0; m < 4; m++)
    for (int n = 0; n < 4; n++) {
      memcpy(out + (m * 4 + n) * n2d, g.data() + (G_GCOV + SY(m, n)) * n2d, sizeof(double) * (size_t)n2d);
      memcpy(out + (16 + m * 4 + n) * n2d, g.data() + (G_GCON + SY(m, n)) * n2d,
             sizeof(double) * (size_t)n2d);
    }
  memcpy(out + 32 * n2d, g.data() + G_GDET * n2d, sizeof(double) * (size_t)n2d);
  memcpy(out + 33 * n2d, g.data() + G_ALPHA * n2d, sizeof(double) * (size_t)n2d);
  return GRMHD_OK;
}

extern "C" int grmhd_set_geometry(grmhd_sim *s, int loc, const double *in) {
  if (!s || !in || loc < 0 || loc > 3) return GRMHD_ERR_INVALID;
  const long long n2d = s->D.n2d;
  if (loc == 3) {
    std::vector<double> c((size_t)(C_NCOMP * n2d));
    for (int l = 0; l < 4; l++)
      for (int m = 0; m < 4; m++)
        for (int n = m; n < 4; n++)
          memcpy(c.data() + (l * 10 + SY(m, n)) * n2d, in + ((l * 4 + m) * 4 + n) * n2d,
                 sizeof(double) * (size_t)n2d);
    CK(cudaMemcpyAsync(s->conn, c.data(), sizeof(double) * c.size(), cudaMemcpyHostToDevice, s->st));
    if (s->connff) launch_to_ff((long long)C_NCOMP * n2d, s->conn, s->connff, s->st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s->st));
    return GRMHD_OK;
  }
  std::vector<double> g((size_t)(G_NCOMP * n2d));
  for (int m = 0; m < 4; m++)
    for (int n = m; n < 4; n++) {
      memcpy(g.data() + (G_GCOV + SY(m, n)) * n2d, in + (m * 4 + n) * n2d, sizeof(double) * (size_t)n2d);
      memcpy(g.data() + (G_GCON + SY(m, n)) * n2d, in + (16 + m * 4 + n) * n2d,
             sizeof(double) * (size_t)n2d);
    }
  memcpy(g.data() + G_GDET * n2d, in + 32 * n2d, sizeof(double) * (size_t)n2d);
  memcpy(g.data() + G_ALPHA * n2d, in + 33 * n2d, sizeof(double) * (size_t)n2d);
  for (long long q = 0; q < n2d; q++) {
    const double al = in[33 * n2d + q];
    g[(size_t)(G_IALPHA * n2d + q)] = 1.0 / al;
    g[(size_t)(G_IGDET * n2d + q)] = 1.0 / in[32 * n2d + q];
    g[(size_t)(G_OMALPHA * n2d + q)] = (1.0 + 1.0 / in[(16 + 0) * n2d + q]) / (1.0 + al);
  }
  CK(cudaMemcpyAsync(s->geom + (long long)loc * G_NCOMP * n2d, g.data(), sizeof(double) * g.size(),
                     cudaMemcpyHostToDevice, s->st));
  if (s->geomf)
    launch_to_f32((long long)G_NCOMP * n2d, s->geom + (long long)loc * G_NCOMP * n2d,
                  s->geomf + (long long)loc * G_NCOMP * n2d, s->st);
  if (s->geomff)  // the whole split copy (its low words follow all locations' high words)
    launch_to_ff((long long)NLOC * G_NCOMP * n2d, s->geom, s->geomff, s->st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s->st));
  return GRMHD_OK;
}

extern "C" int grmhd_divb(grmhd_sim *s, double *divb_max, double *gb_max) {
  if (!s || !divb_max) return GRMHD_ERR_INVALID;
  // the two result words live in the (between-step) EMF scratch
  unsigned long long *dev = (unsigned long long *)s->emf, host[2];
  launch_divb(s->A, s->P, dev, s->st);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(host, dev, sizeof(host), cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  memcpy(divb_max, &host[0], sizeof(double));
  if (gb_max) memcpy(gb_max, &host[1], sizeof(double));
  return GRMHD_OK;
}

extern "C" int grmhd_autotune(grmhd_sim *s, int trials, double *ms_before, double *ms_after) {
  if (!s || trials < 1) return GRMHD_ERR_INVALID;
  sim_drop_graph(s);  // the launch shapes may change
  return plan_autotune(s->plan, trials, s->st, ms_before, ms_after);
}

extern "C" int grmhd_set_recon_walk(grmhd_sim *s, int zones_per_thread, int *chosen) {
  if (!s) return GRMHD_ERR_INVALID;
  sim_drop_graph(s);  // the launch shapes change
  const int rc = plan_set_rwalk(s->plan, zones_per_thread);
  if (rc == GRMHD_OK && chosen) *chosen = s->plan.host_items[0].A.rwalk;
  return rc;
}

extern "C" int grmhd_profile(grmhd_sim *s, int enable) {
  if (!s) return GRMHD_ERR_INVALID;
  s->prof_on = enable ? 1 : 0;
  return GRMHD_OK;
}

extern "C" int grmhd_get_profile(grmhd_sim *s, grmhd_profile_data *out, int reset) {
  if (!s || !out) return GRMHD_ERR_INVALID;
  CK(cudaStreamSynchronize(s->st));
  collect_profile(s);
  for (int c = 0; c < GRMHD_NKCLASS; c++) {
    out->ms[c] = s->prof_ms[c];
    out->launches[c] = s->launches[c];
  }
  if (reset) {
    for (int c = 0; c < GRMHD_NKCLASS; c++) {
      s->prof_ms[c] = 0.0;
      s->launches[c] = 0;
    }
  }
  return GRMHD_OK;
}

extern "C" const char *grmhd_strerror(int code) {
  switch (code) {
    case GRMHD_OK: return "ok";
    case GRMHD_ERR_INVALID: return "invalid argument";
    case GRMHD_ERR_NOMEM: return "device allocation failed";
    case GRMHD_ERR_CUDA: return "CUDA runtime error";
    case GRMHD_ERR_INVERSION: return "failed zone with no valid neighbour";
    case GRMHD_ERR_DT: return "no finite time step";
    default: return "unknown error";
  }
}
