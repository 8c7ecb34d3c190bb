// server.cu -- the serving request loop (grmhd_server_* in include/grmhd.h).
//
// One host thread per server owns every device object it creates.  Callers
// submit simulations from any thread; the loop moves them through
//   incoming (submitted) -> pending (FIFO, waiting for HBM) -> active
//   (state resident, stepped in rounds) -> done (result in host memory),
// each active simulation on its own CUDA stream so that uploads and
// downloads of one simulation do not wait for the others' work.  A round
// is one batch step of all active simulations: every kernel of the cycle
// is one launch over all of them (plan.h), and the batch is rebuilt only
// when a simulation joins or leaves.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/grmhd.h"

namespace {

struct Request {
  long long id;
  grmhd_grid grid;
  grmhd_metric metric;
  grmhd_params params;
  const double *P_in;
  double *P_out;
  const double *K_in;  // electron entropies (requests with electrons), same ghosts as P
  double *K_out;
  int in_ghosts, out_ghosts;
  long long nsteps, remaining;
  size_t bytes;
  long long zones;
  double t_arrival, t_admit, t_done;
  int status;
  grmhd_stats stats;
  grmhd_sim *sim;
  cudaStream_t st;
};

}  // namespace

struct grmhd_server {
  grmhd_server_config cfg;
  int device;
  std::chrono::steady_clock::time_point t0;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv;       // loop: new submissions or stop
  std::condition_variable cv_done;  // callers: results or idle
  bool stop;
  std::deque<Request *> incoming;  // guarded by mu
  std::deque<Request *> done;      // guarded by mu
  // owned by the loop thread
  std::deque<Request *> pending;
  std::vector<Request *> active;
  grmhd_batch *batch;
  bool batch_dirty;
  // statistics, guarded by mu
  long long submitted, completed, failed, rounds, launches, in_flight;
  double zone_cycles, busy;
  size_t used, peak_bytes;
  int n_active, n_pending, peak_active;
};

static double now_s(const grmhd_server *s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

extern "C" double grmhd_server_now(grmhd_server *s) { return s ? now_s(s) : 0.0; }

// Finish a request (result or error): free its device objects, publish it.
static void finish(grmhd_server *s, Request *r, int status) {
  if (r->sim) grmhd_destroy(r->sim);
  r->sim = nullptr;
  if (r->st) cudaStreamDestroy(r->st);
  r->st = nullptr;
  r->status = status;
  r->t_done = now_s(s);
  std::lock_guard<std::mutex> lk(s->mu);
  s->used -= r->t_admit >= 0.0 ? r->bytes : 0;
  if (status == GRMHD_OK || status == GRMHD_ERR_INVERSION)
    s->completed++;
  else
    s->failed++;
  s->in_flight--;
  s->done.push_back(r);
  s->cv_done.notify_all();
}

// Admit waiting requests while they fit: FIFO takes the oldest until one
// does not fit; SWF takes, repeatedly, the smallest-work request that fits.
static void admit(grmhd_server *s) {
  long long zones = 0;
  for (Request *r : s->active) zones += r->zones;
  for (;;) {
    if (s->pending.empty()) break;
    size_t used;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      used = s->used;
    }
    auto fits = [&](const Request *r) {
      if (used + r->bytes > s->cfg.hbm_budget) return false;
      return !(s->cfg.max_active_zones > 0 && !s->active.empty() &&
               zones + r->zones > s->cfg.max_active_zones);
    };
    std::deque<Request *>::iterator pick = s->pending.end();
    if (s->cfg.policy == GRMHD_SERVE_SWF) {
      double best = 0.0;
      for (auto it = s->pending.begin(); it != s->pending.end(); ++it) {
        const double w = (double)(*it)->zones * (double)(*it)->nsteps;
        if (fits(*it) && (pick == s->pending.end() || w < best)) {
          pick = it;
          best = w;
        }
      }
    } else if (fits(s->pending.front())) {
      pick = s->pending.begin();
    }
    if (pick == s->pending.end()) break;
    Request *r = *pick;
    s->pending.erase(pick);
    int rc = (cudaStreamCreateWithFlags(&r->st, cudaStreamNonBlocking) == cudaSuccess)
                 ? GRMHD_OK
                 : GRMHD_ERR_CUDA;
    if (rc == GRMHD_OK) rc = grmhd_create(&r->grid, &r->metric, &r->params, r->st, &r->sim);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (rc == GRMHD_OK) {
        s->used += r->bytes;
        s->peak_bytes = std::max(s->peak_bytes, s->used);
      }
    }
    r->t_admit = (rc == GRMHD_OK) ? 0.0 : -1.0;  // marks the bytes as held
    if (rc == GRMHD_OK)
      rc = r->in_ghosts ? grmhd_set_prims_ghost(r->sim, r->P_in, 0) : grmhd_set_prims(r->sim, r->P_in, 0);
    if (rc == GRMHD_OK && r->K_in) rc = grmhd_set_electrons(r->sim, r->K_in, r->in_ghosts, 0);
    if (rc != GRMHD_OK) {
      finish(s, r, rc);
      continue;
    }
    r->t_admit = now_s(s);
    s->active.push_back(r);
    zones += r->zones;
    s->batch_dirty = true;
  }
}

// One round over the active set: a batch step of q cycles, then the
// results of the simulations that have taken all their cycles.
static void round_once(grmhd_server *s) {
  if (s->batch_dirty) {
    if (s->batch) grmhd_batch_destroy(s->batch);
    s->batch = nullptr;
    std::vector<grmhd_sim *> sims;
    for (Request *r : s->active) sims.push_back(r->sim);
    const int rc = grmhd_batch_create(sims.data(), (int)sims.size(), &s->batch);
    if (rc != GRMHD_OK) {
      for (Request *r : s->active) finish(s, r, rc);
      s->active.clear();
      return;
    }
    s->batch_dirty = false;
  }
  long long q = s->cfg.quantum;
  for (Request *r : s->active) q = std::min(q, r->remaining);
  const double t_start = now_s(s);
  int rc = grmhd_batch_step(s->batch, (int)q, s->cfg.use_graph);
  if (rc == GRMHD_OK) rc = grmhd_batch_sync(s->batch);
  grmhd_batch_info info;
  memset(&info, 0, sizeof(info));
  grmhd_batch_get_info(s->batch, &info);
  double zc = 0.0;
  for (Request *r : s->active) zc += (double)r->zones * (double)q;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->busy += now_s(s) - t_start;
    s->rounds++;
    s->launches += (long long)info.launches_per_step * q;
    if (rc == GRMHD_OK) s->zone_cycles += zc;
  }
  if (rc != GRMHD_OK) {
    grmhd_batch_destroy(s->batch);
    s->batch = nullptr;
    for (Request *r : s->active) finish(s, r, rc);
    s->active.clear();
    return;
  }
  std::vector<Request *> keep, fin;
  for (Request *r : s->active) {
    r->remaining -= q;
    (r->remaining > 0 ? keep : fin).push_back(r);
  }
  if (fin.empty()) return;
  // the batch references the finishing simulations: drop it first
  grmhd_batch_destroy(s->batch);
  s->batch = nullptr;
  s->batch_dirty = true;
  s->active = keep;
  for (Request *r : fin) {
    int frc = grmhd_get_prims(r->sim, r->P_out, r->out_ghosts, 0);
    if (frc == GRMHD_OK && r->K_out) frc = grmhd_get_electrons(r->sim, r->K_out, r->out_ghosts, 0);
    if (frc == GRMHD_OK) frc = grmhd_step(r->sim, 0, &r->stats);  // statistics + failure check
    finish(s, r, frc);
  }
}

static void loop(grmhd_server *s) {
  cudaSetDevice(s->device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->pending.empty() && s->active.empty() && s->incoming.empty() && !s->stop)
        s->cv.wait(lk, [&] { return s->stop || !s->incoming.empty(); });
      if (s->stop) break;
      while (!s->incoming.empty()) {
        s->pending.push_back(s->incoming.front());
        s->incoming.pop_front();
      }
    }
    admit(s);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->n_active = (int)s->active.size();
      s->n_pending = (int)s->pending.size();
      s->peak_active = std::max(s->peak_active, s->n_active);
    }
    if (!s->active.empty()) round_once(s);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->n_active = (int)s->active.size();
      s->n_pending = (int)s->pending.size();
      if (s->in_flight == 0) s->cv_done.notify_all();
    }
  }
  // stopped: drop what is left
  if (s->batch) grmhd_batch_destroy(s->batch);
  s->batch = nullptr;
  for (Request *r : s->active) {
    if (r->sim) grmhd_destroy(r->sim);
    if (r->st) cudaStreamDestroy(r->st);
    delete r;
  }
  s->active.clear();
  for (Request *r : s->pending) delete r;
  s->pending.clear();
}

extern "C" int grmhd_server_create(const grmhd_server_config *cfg, grmhd_server **out) {
  if (!out) return GRMHD_ERR_INVALID;
  *out = nullptr;
  grmhd_server_config c;
  if (cfg) {
    c = *cfg;
  } else {
    memset(&c, 0, sizeof(c));
    c.quantum = 8;
    c.use_graph = 1;
  }
  if (c.quantum < 1 || c.max_active_zones < 0) return GRMHD_ERR_INVALID;
  if (c.policy != GRMHD_SERVE_FIFO && c.policy != GRMHD_SERVE_SWF) return GRMHD_ERR_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GRMHD_ERR_CUDA;
  if (c.hbm_budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return GRMHD_ERR_CUDA;
    c.hbm_budget = fr / 10 * 9;
  }
  grmhd_server *s = new (std::nothrow) grmhd_server();
  if (!s) return GRMHD_ERR_NOMEM;
  s->cfg = c;
  s->device = dev;
  s->t0 = std::chrono::steady_clock::now();
  s->stop = false;
  s->batch = nullptr;
  s->batch_dirty = true;
  s->submitted = s->completed = s->failed = s->rounds = s->launches = s->in_flight = 0;
  s->zone_cycles = s->busy = 0.0;
  s->used = s->peak_bytes = 0;
  s->n_active = s->n_pending = s->peak_active = 0;
  try {
    s->th = std::thread(loop, s);
  } catch (...) {
    delete s;
    return GRMHD_ERR_NOMEM;
  }
  *out = s;
  return GRMHD_OK;
}

static int submit(grmhd_server *s, long long id, const grmhd_grid *grid,
                  const grmhd_metric *metric, const grmhd_params *params, const double *P_in,
                  int in_ghosts, double *P_out, int out_ghosts, const double *K_in, double *K_out,
                  long long nsteps, double t_arrival) {
  if (!s || !grid || !metric || !params || !P_in || !P_out || nsteps < 1 || nsteps > (1ll << 30))
    return GRMHD_ERR_INVALID;
  // the electron entropies come and go with the request exactly when it evolves them
  const bool elec = params->electrons.model != GRMHD_ELEC_OFF;
  if (elec != (K_in != nullptr) || elec != (K_out != nullptr)) return GRMHD_ERR_INVALID;
  size_t bytes = 0;
  const int rc = grmhd_footprint(grid, metric, params, &bytes);
  if (rc != GRMHD_OK) return rc;
  if (bytes > s->cfg.hbm_budget) return GRMHD_ERR_NOMEM;
  Request *r = new (std::nothrow) Request();
  if (!r) return GRMHD_ERR_NOMEM;
  memset(r, 0, sizeof(*r));
  r->id = id;
  r->grid = *grid;
  r->metric = *metric;
  r->params = *params;
  r->P_in = P_in;
  r->P_out = P_out;
  r->K_in = K_in;
  r->K_out = K_out;
  r->in_ghosts = in_ghosts ? 1 : 0;
  r->out_ghosts = out_ghosts ? 1 : 0;
  r->nsteps = r->remaining = nsteps;
  r->bytes = bytes;
  r->zones = (long long)grid->n1 * grid->n2 * grid->n3;
  r->t_arrival = t_arrival < 0.0 ? now_s(s) : t_arrival;
  r->t_admit = -1.0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->incoming.push_back(r);
    s->submitted++;
    s->in_flight++;
  }
  s->cv.notify_all();
  return GRMHD_OK;
}

extern "C" int grmhd_server_submit(grmhd_server *s, long long id, const grmhd_grid *grid,
                                   const grmhd_metric *metric, const grmhd_params *params,
                                   const double *P_in, int in_ghosts, double *P_out,
                                   int out_ghosts, long long nsteps, double t_arrival) {
  return submit(s, id, grid, metric, params, P_in, in_ghosts, P_out, out_ghosts, nullptr, nullptr,
                nsteps, t_arrival);
}

extern "C" int grmhd_server_submit_electrons(grmhd_server *s, long long id, const grmhd_grid *grid,
                                             const grmhd_metric *metric,
                                             const grmhd_params *params, const double *P_in,
                                             const double *K_in, int in_ghosts, double *P_out,
                                             double *K_out, int out_ghosts, long long nsteps,
                                             double t_arrival) {
  return submit(s, id, grid, metric, params, P_in, in_ghosts, P_out, out_ghosts, K_in, K_out,
                nsteps, t_arrival);
}

extern "C" int grmhd_server_poll(grmhd_server *s, grmhd_server_result *res, int max, int wait_ms) {
  if (!s || !res || max < 0) return GRMHD_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && wait_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
  int n = 0;
  while (n < max && !s->done.empty()) {
    Request *r = s->done.front();
    s->done.pop_front();
    grmhd_server_result &o = res[n++];
    o.id = r->id;
    o.status = r->status;
    o.zones = r->zones;
    o.steps = r->nsteps - r->remaining;
    o.t_arrival = r->t_arrival;
    o.t_admit = r->t_admit;
    o.t_done = r->t_done;
    o.stats = r->stats;
    delete r;
  }
  return n;
}

extern "C" int grmhd_server_drain(grmhd_server *s, int timeout_ms) {
  if (!s) return GRMHD_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  auto idle = [&] { return s->in_flight == 0; };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, idle);
    return GRMHD_OK;
  }
  return s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), idle) ? GRMHD_OK
                                                                               : GRMHD_ERR_CUDA;
}

extern "C" int grmhd_server_get_stats(grmhd_server *s, grmhd_server_stats *o) {
  if (!s || !o) return GRMHD_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  o->now = now_s(s);
  o->submitted = s->submitted;
  o->completed = s->completed;
  o->failed = s->failed;
  o->rounds = s->rounds;
  o->zone_cycles = s->zone_cycles;
  o->busy_seconds = s->busy;
  o->bytes_in_use = s->used;
  o->peak_bytes = s->peak_bytes;
  o->budget = s->cfg.hbm_budget;
  o->active = s->n_active;
  o->pending = s->n_pending + (int)s->incoming.size();
  o->peak_active = s->peak_active;
  o->launches = s->launches;
  return GRMHD_OK;
}

extern "C" int grmhd_server_destroy(grmhd_server *s) {
  if (!s) return GRMHD_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->th.joinable()) s->th.join();
  for (Request *r : s->incoming) delete r;
  for (Request *r : s->done) delete r;
  delete s;
  return GRMHD_OK;
}
