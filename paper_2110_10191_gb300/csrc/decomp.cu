// decomp.cu -- a grid decomposed into blocks (grmhd_decomp_* in
// include/grmhd.h): the paper's domain decomposition ("Scaling" section;
// one mesh block per node), on one GPU.
//
// Each block is a simulation of its part of the global grid (its geometry
// computed from global zone indices, its physical boundaries where the
// global grid has them); all blocks advance together as one launch plan.
// What a single grid gets from its own ghost fill, a block gets from its
// neighbours by an exchange of edge zones, in the order of the single
// grid's fill (X1 ghosts of interior rows, then X2 ghosts of every column,
// then X3), so every ghost zone holds the value the undecomposed grid holds
// there.  The signal-speed maxima are combined over the blocks before the
// time step, and before the fixup the first layer of primitives and failure
// flags is exchanged, so a failed zone at a block edge averages over the
// same neighbours as in the undecomposed grid.  Blocks that evolve the
// electron entropies exchange them with the primitives in both.  The evolution is therefore
// bitwise independent of the decomposition (the paper's decomposition
// tests, end of its "Tests" section).
#include <cstring>
#include <new>
#include <vector>

#include "../../include/grmhd.h"
#include "grmhd_impl.h"
#include "plan.h"
#include "sim_impl.h"
#include "step_bodies.cuh"

using namespace grmhd;

namespace {

// one copy box: destination zones lo..lo+ext of block dst from block src at
// index + shift
struct XDesc {
  int dst, src;
  int lo[3], ext[3], shift[3];
  int nvars;  // primitives copied (the first nvars)
  int flag;   // 1: the failure flags too
  int kvars;  // electron entropies copied (blocks that evolve them: 2)
};

__global__ void kx_exchange(const StageItem *__restrict__ items, const XDesc *__restrict__ desc,
                            const int *__restrict__ map, const int *__restrict__ loc, int which) {
  const XDesc &x = desc[__ldg(map + blockIdx.x)];
  const long long t = (long long)__ldg(loc + blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= (long long)x.ext[0] * x.ext[1] * x.ext[2]) return;
  const int i = x.lo[0] + (int)(t % x.ext[0]);
  const int j = x.lo[1] + (int)((t / x.ext[0]) % x.ext[1]);
  const int k = x.lo[2] + (int)(t / ((long long)x.ext[0] * x.ext[1]));
  const StageItem &d = items[x.dst], &s = items[x.src];
  const long long cd = zid(d.A.D, i, j, k);
  const long long cs = zid(s.A.D, i + x.shift[0], j + x.shift[1], k + x.shift[2]);
  double *Pd = which ? d.Ph : d.P;
  const double *Ps = which ? s.Ph : s.P;
  for (int v = 0; v < x.nvars; v++) Pd[v * d.A.D.ntot + cd] = Ps[v * s.A.D.ntot + cs];
  if (x.flag) d.pflag[cd] = s.pflag[cs];
  if (x.kvars) {
    double *Kd = which ? d.Kh : d.K;
    const double *Ks = which ? s.Kh : s.K;
    for (int q = 0; q < x.kvars; q++) Kd[q * d.A.D.ntot + cd] = Ks[q * s.A.D.ntot + cs];
  }
}

// the signal-speed maxima of all blocks, given to every block
__global__ void kx_ctop_reduce(const StageItem *__restrict__ items, int n) {
  const int d = threadIdx.x;
  if (d >= 3) return;
  unsigned long long m = 0ull;
  for (int g = 0; g < n; g++) {
    const unsigned long long b = items[g].A.clk->ctop_bits[d];
    m = (b > m) ? b : m;
  }
  for (int g = 0; g < n; g++) items[g].A.clk->ctop_bits[d] = m;
}

// device tables of one exchange pass
struct XTable {
  XDesc *desc = nullptr;
  int *map = nullptr, *loc = nullptr;
  int nblocks = 0;
};

}  // namespace

struct grmhd_decomp {
  int nb[3];
  grmhd_grid grid;
  grmhd_metric metric;
  grmhd_params params;
  cudaStream_t st;
  std::vector<grmhd_sim *> blocks;  // index bx + nb0 (by + nb1 bz)
  std::vector<BlockSpec> spec;
  Plan plan;
  XTable full[3], layer[3];  // ghost fill (3 layers, 8 primitives) / fixup (1 layer, 5 + flags)
  unsigned long long unrec_seen, dterr_seen;
};

static void xtable_free(XTable &t) {
  if (t.desc) cudaFree(t.desc);
  if (t.map) cudaFree(t.map);
  if (t.loc) cudaFree(t.loc);
  t = XTable();
}

static void decomp_free(grmhd_decomp *dc) {
  for (int p = 0; p < 3; p++) {
    xtable_free(dc->full[p]);
    xtable_free(dc->layer[p]);
  }
  plan_free(dc->plan);
  for (grmhd_sim *s : dc->blocks)
    if (s) grmhd_destroy(s);
  dc->blocks.clear();
}

static int xtable_build(XTable &t, const std::vector<XDesc> &d) {
  std::vector<int> map, loc;
  for (size_t q = 0; q < d.size(); q++) {
    const long long nz = (long long)d[q].ext[0] * d[q].ext[1] * d[q].ext[2];
    for (long long b = 0; b < (nz + BS - 1) / BS; b++) {
      map.push_back((int)q);
      loc.push_back((int)b);
    }
  }
  t.nblocks = (int)map.size();
  if (d.empty()) return GRMHD_OK;
  if (cudaMalloc(&t.desc, sizeof(XDesc) * d.size()) != cudaSuccess ||
      cudaMalloc(&t.map, sizeof(int) * map.size()) != cudaSuccess ||
      cudaMalloc(&t.loc, sizeof(int) * loc.size()) != cudaSuccess) {
    cudaGetLastError();
    return GRMHD_ERR_NOMEM;
  }
  if (cudaMemcpy(t.desc, d.data(), sizeof(XDesc) * d.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(t.map, map.data(), sizeof(int) * map.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(t.loc, loc.data(), sizeof(int) * loc.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return GRMHD_ERR_CUDA;
  return GRMHD_OK;
}

static int exchange(const grmhd_decomp *dc, const XTable &t, int which) {
  if (t.nblocks == 0) return 0;
  kx_exchange<<<t.nblocks, BS, 0, dc->st>>>(dc->plan.items, t.desc, t.map, t.loc, which);
  return 1;
}

// The ghost fill of array `which` over all blocks: per pass, the physical
// boundaries, then the edges of the neighbours.
static int fill(const grmhd_decomp *dc, int which) {
  int nl = 0;
  for (int p = 0; p < 3; p++) {
    nl += plan_bounds_pass(dc->plan, which, p, dc->st, nullptr);
    nl += exchange(dc, dc->full[p], which);
  }
  return nl;
}

static int bidx(const grmhd_decomp *dc, int bx, int by, int bz) {
  return bx + dc->nb[0] * (by + dc->nb[1] * bz);
}

extern "C" int grmhd_decomp_create(const grmhd_grid *grid, const grmhd_metric *metric,
                                   const grmhd_params *params, const int nblocks[3], void *stream,
                                   grmhd_decomp **out) {
  if (!out || !nblocks) return GRMHD_ERR_INVALID;
  *out = nullptr;
  Dims G;
  int rc = validate_problem(grid, metric, params, &G);
  if (rc != GRMHD_OK) return rc;
  for (int d = 0; d < 3; d++) {
    if (nblocks[d] < 1 || nblocks[d] > G.n[d]) return GRMHD_ERR_INVALID;
    if (nblocks[d] > 1 && G.n[d] / nblocks[d] < NG) return GRMHD_ERR_INVALID;  // blocks >= NG zones
    if (nblocks[d] > 1 && params->bc[d][0] == GRMHD_BC_POLAR && G.n[d] / nblocks[d] < NG)
      return GRMHD_ERR_INVALID;
  }
  grmhd_decomp *dc = new (std::nothrow) grmhd_decomp();
  if (!dc) return GRMHD_ERR_NOMEM;
  for (int d = 0; d < 3; d++) dc->nb[d] = nblocks[d];
  dc->grid = *grid;
  dc->metric = *metric;
  dc->params = *params;
  dc->st = (cudaStream_t)stream;
  const int nblk = nblocks[0] * nblocks[1] * nblocks[2];
  // block extents: as equal as possible, the larger first
  std::vector<int> off[3], len[3];
  for (int d = 0; d < 3; d++)
    for (int b = 0, o = 0; b < nblocks[d]; b++) {
      const int l = G.n[d] / nblocks[d] + (b < G.n[d] % nblocks[d] ? 1 : 0);
      off[d].push_back(o);
      len[d].push_back(l);
      o += l;
    }
  dc->spec.resize(nblk);
  dc->blocks.assign(nblk, nullptr);
  std::vector<StageItem> items(nblk);
  for (int bz = 0; bz < nblocks[2]; bz++)
    for (int by = 0; by < nblocks[1]; by++)
      for (int bx = 0; bx < nblocks[0]; bx++) {
        const int b = bidx(dc, bx, by, bz);
        const int c[3] = {bx, by, bz};
        BlockSpec &sp = dc->spec[b];
        grmhd_params bp = *params;
        for (int d = 0; d < 3; d++) {
          sp.off[d] = off[d][c[d]];
          sp.n[d] = len[d][c[d]];
          const bool split = nblocks[d] > 1;
          const bool periodic = params->bc[d][0] == GRMHD_BC_PERIODIC;
          // a side is shared when a neighbour block lies beyond it, across the
          // periodic seam too; the fixup looks across it only inside the
          // global grid (the whole grid's fixup averages over its own zones,
          // not over the periodic images in its ghosts)
          const bool xl = split && (c[d] > 0 || periodic), xh = split && (c[d] < nblocks[d] - 1 || periodic);
          sp.xlo[d] = split && c[d] > 0;
          sp.xhi[d] = split && c[d] < nblocks[d] - 1;
          if (xl) bp.bc[d][0] = BC_EXCHANGE;
          if (xh) bp.bc[d][1] = BC_EXCHANGE;
        }
        rc = sim_create(grid, metric, &bp, stream, &sp, &dc->blocks[b]);
        if (rc != GRMHD_OK) {
          decomp_free(dc);
          delete dc;
          return rc;
        }
        if (cudaMemcpy(&items[b], dc->blocks[b]->plan.items, sizeof(StageItem),
                       cudaMemcpyDeviceToHost) != cudaSuccess) {
          decomp_free(dc);
          delete dc;
          return GRMHD_ERR_CUDA;
        }
      }
  rc = plan_build(dc->plan, items.data(), nblk);
  // exchange boxes per pass and side
  std::vector<XDesc> full[3], layer[3];
  for (int bz = 0; bz < nblocks[2] && rc == GRMHD_OK; bz++)
    for (int by = 0; by < nblocks[1]; by++)
      for (int bx = 0; bx < nblocks[0]; bx++) {
        const int b = bidx(dc, bx, by, bz);
        const int c[3] = {bx, by, bz};
        const BlockSpec &sp = dc->spec[b];
        const int s[3] = {sp.n[0] + 2 * NG, sp.n[1] + 2 * NG, sp.n[2] + 2 * NG};
        grmhd_sim *self = dc->blocks[b];
        for (int d = 0; d < 3; d++)
          for (int side = 0; side < 2; side++) {
            if (self->A.bc[d][side] != BC_EXCHANGE) continue;
            int cn[3] = {c[0], c[1], c[2]};
            cn[d] = (c[d] + (side ? 1 : -1) + nblocks[d]) % nblocks[d];
            const int src = bidx(dc, cn[0], cn[1], cn[2]);
            const int nsrc = dc->spec[src].n[d];
            for (int kind = 0; kind < 2; kind++) {  // 0: full ghost fill, 1: fixup layer
              XDesc x;
              memset(&x, 0, sizeof(x));
              x.dst = b;
              x.src = src;
              const int depth = kind ? 1 : NG;
              for (int e = 0; e < 3; e++) {
                // transverse range: earlier passes' ghosts included, later ones not
                if (e < d) {
                  x.lo[e] = kind ? NG - 1 : 0;
                  x.ext[e] = kind ? sp.n[e] + 2 : s[e];
                } else if (e > d) {
                  x.lo[e] = NG;
                  x.ext[e] = sp.n[e];
                }
              }
              x.lo[d] = side ? sp.n[d] + NG : NG - depth;
              x.ext[d] = depth;
              x.shift[d] = side ? -sp.n[d] : nsrc;
              x.nvars = kind ? 5 : NV;
              x.flag = kind;
              x.kvars = params->electrons.model != GRMHD_ELEC_OFF ? 2 : 0;
              (kind ? layer : full)[d].push_back(x);
            }
          }
      }
  for (int p = 0; p < 3 && rc == GRMHD_OK; p++) {
    rc = xtable_build(dc->full[p], full[p]);
    if (rc == GRMHD_OK) rc = xtable_build(dc->layer[p], layer[p]);
  }
  if (rc != GRMHD_OK) {
    decomp_free(dc);
    delete dc;
    return rc;
  }
  *out = dc;
  return GRMHD_OK;
}

extern "C" int grmhd_decomp_destroy(grmhd_decomp *dc) {
  if (!dc) return GRMHD_OK;
  cudaStreamSynchronize(dc->st);
  decomp_free(dc);
  delete dc;
  return GRMHD_OK;
}

// The global array of nvar variables (interior or with ghosts) into the
// blocks' stage array 0 (the primitives, or the electron entropies with
// elec), then the ghost fill.
static int set_global(grmhd_decomp *dc, const double *P, int with_ghosts, bool elec) {
  const int nvar = elec ? 2 : NV;
  const int gn[3] = {dc->grid.n1, dc->grid.n2, dc->grid.n3};
  const long long gs0 = gn[0] + 2 * NG, gs1 = gn[1] + 2 * NG, gs2 = gn[2] + 2 * NG;
  const long long gtot = gs0 * gs1 * gs2;
  // the global array with ghosts (interior input: ghosts left to the fill)
  std::vector<double> g;
  const double *src = P;
  if (!with_ghosts) {
    g.assign((size_t)(nvar * gtot), 0.0);
    const long long nz = (long long)gn[0] * gn[1] * gn[2];
    for (int v = 0; v < nvar; v++)
      for (int k = 0; k < gn[2]; k++)
        for (int j = 0; j < gn[1]; j++)
          memcpy(&g[(size_t)(v * gtot + ((k + NG) * gs1 + j + NG) * gs0 + NG)],
                 P + v * nz + ((long long)k * gn[1] + j) * gn[0], sizeof(double) * gn[0]);
    src = g.data();
  }
  for (size_t b = 0; b < dc->blocks.size(); b++) {
    grmhd_sim *s = dc->blocks[b];
    const BlockSpec &sp = dc->spec[b];
    const Dims &D = s->D;
    std::vector<double> h((size_t)(nvar * D.ntot));
    for (int v = 0; v < nvar; v++)
      for (int k = 0; k < D.s[2]; k++)
        for (int j = 0; j < D.s[1]; j++)
          memcpy(&h[(size_t)(v * D.ntot + ((long long)k * D.s[1] + j) * D.s[0])],
                 src + v * gtot + ((long long)(k + sp.off[2]) * gs1 + (j + sp.off[1])) * gs0 + sp.off[0],
                 sizeof(double) * D.s[0]);
    if (cudaMemcpyAsync(elec ? s->K : s->P, h.data(), sizeof(double) * h.size(),
                        cudaMemcpyHostToDevice, dc->st) != cudaSuccess ||
        cudaStreamSynchronize(dc->st) != cudaSuccess)
      return GRMHD_ERR_CUDA;
  }
  fill(dc, 0);
  // the ghosts of a fixed side keep their set values in both stage arrays
  for (grmhd_sim *s : dc->blocks) {
    if (cudaMemcpyAsync(s->Ph, s->P, sizeof(double) * NV * (size_t)s->D.ntot, cudaMemcpyDeviceToDevice,
                        dc->st) != cudaSuccess)
      return GRMHD_ERR_CUDA;
    if (s->K && cudaMemcpyAsync(s->Kh, s->K, sizeof(double) * 2 * (size_t)s->D.ntot,
                                cudaMemcpyDeviceToDevice, dc->st) != cudaSuccess)
      return GRMHD_ERR_CUDA;
  }
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(dc->st) != cudaSuccess)
    return GRMHD_ERR_CUDA;
  return GRMHD_OK;
}

// The blocks' stage array 0 (primitives or electron entropies) as the
// global array, interior or with ghosts.
static int get_global(grmhd_decomp *dc, double *P, int with_ghosts, bool elec) {
  const int nvar = elec ? 2 : NV;
  const int gn[3] = {dc->grid.n1, dc->grid.n2, dc->grid.n3};
  const long long gs[3] = {gn[0] + 2 * NG, gn[1] + 2 * NG, gn[2] + 2 * NG};
  const long long gtot = gs[0] * gs[1] * gs[2], nz = (long long)gn[0] * gn[1] * gn[2];
  for (size_t b = 0; b < dc->blocks.size(); b++) {
    grmhd_sim *s = dc->blocks[b];
    const BlockSpec &sp = dc->spec[b];
    const Dims &D = s->D;
    std::vector<double> h((size_t)(nvar * D.ntot));
    if (cudaMemcpyAsync(h.data(), elec ? s->K : s->P, sizeof(double) * h.size(),
                        cudaMemcpyDeviceToHost, dc->st) != cudaSuccess ||
        cudaStreamSynchronize(dc->st) != cudaSuccess)
      return GRMHD_ERR_CUDA;
    // the zones this block owns: its interior, and the global ghosts beyond
    // its outer sides
    int lo[3], hi[3];
    const int c[3] = {(int)(b % dc->nb[0]), (int)((b / dc->nb[0]) % dc->nb[1]),
                      (int)(b / (dc->nb[0] * dc->nb[1]))};
    for (int d = 0; d < 3; d++) {
      lo[d] = (with_ghosts && c[d] == 0) ? 0 : NG;
      hi[d] = (with_ghosts && c[d] == dc->nb[d] - 1) ? sp.n[d] + 2 * NG : sp.n[d] + NG;
    }
    for (int v = 0; v < nvar; v++)
      for (int k = lo[2]; k < hi[2]; k++)
        for (int j = lo[1]; j < hi[1]; j++) {
          const double *row = &h[(size_t)(v * D.ntot + ((long long)k * D.s[1] + j) * D.s[0] + lo[0])];
          const long long gk = k + sp.off[2], gj = j + sp.off[1], gi = lo[0] + sp.off[0];
          double *dst = with_ghosts ? P + v * gtot + (gk * gs[1] + gj) * gs[0] + gi
                                    : P + v * nz + ((gk - NG) * gn[1] + (gj - NG)) * gn[0] + (gi - NG);
          memcpy(dst, row, sizeof(double) * (hi[0] - lo[0]));
        }
  }
  return GRMHD_OK;
}

extern "C" int grmhd_decomp_set_prims(grmhd_decomp *dc, const double *P, int with_ghosts) {
  if (!dc || !P) return GRMHD_ERR_INVALID;
  return set_global(dc, P, with_ghosts, false);
}

extern "C" int grmhd_decomp_get_prims(grmhd_decomp *dc, double *P, int with_ghosts) {
  if (!dc || !P) return GRMHD_ERR_INVALID;
  return get_global(dc, P, with_ghosts, false);
}

extern "C" int grmhd_decomp_set_electrons(grmhd_decomp *dc, const double *K, int with_ghosts) {
  if (!dc || !K || dc->params.electrons.model == GRMHD_ELEC_OFF) return GRMHD_ERR_INVALID;
  return set_global(dc, K, with_ghosts, true);
}

extern "C" int grmhd_decomp_get_electrons(grmhd_decomp *dc, double *K, int with_ghosts) {
  if (!dc || !K || dc->params.electrons.model == GRMHD_ELEC_OFF) return GRMHD_ERR_INVALID;
  return get_global(dc, K, with_ghosts, true);
}

extern "C" int grmhd_decomp_step(grmhd_decomp *dc, int nsteps, grmhd_stats *stats) {
  if (!dc || nsteps < 0) return GRMHD_ERR_INVALID;
  const Plan &p = dc->plan;
  cudaStream_t st = dc->st;
  for (int n = 0; n < nsteps; n++)
    for (int stage = 0; stage < 2; stage++) {
      const int in = stage, out = 1 - stage;
      plan_fluxes(p, in, st, nullptr);
      if (stage == 0) {
        kx_ctop_reduce<<<1, 32, 0, st>>>(p.items, p.ngrid);
        plan_clock(p, 1, st, nullptr);
      }
      plan_fix_ct(p, st, nullptr);
      plan_update_only(p, in, stage ? 1.0 : 0.5, stage ? 2 : 1, st, nullptr);
      for (int q = 0; q < 3; q++) exchange(dc, dc->layer[q], out);
      plan_fixup(p, out, st, nullptr);
      fill(dc, out);
      if (stage == 1) plan_clock(p, 2, st, nullptr);
    }
  if (cudaGetLastError() != cudaSuccess) return GRMHD_ERR_CUDA;
  if (!stats) return GRMHD_OK;
  return grmhd_decomp_get_stats(dc, stats, 1);
}

extern "C" int grmhd_decomp_get_stats(grmhd_decomp *dc, grmhd_stats *out, int check) {
  if (!dc || !out) return GRMHD_ERR_INVALID;
  if (cudaStreamSynchronize(dc->st) != cudaSuccess) return GRMHD_ERR_CUDA;
  memset(out, 0, sizeof(*out));
  unsigned long long unrec = 0, dterr = 0;
  for (size_t b = 0; b < dc->blocks.size(); b++) {
    Clock c;
    if (cudaMemcpy(&c, dc->blocks[b]->clk, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess)
      return GRMHD_ERR_CUDA;
    if (b == 0) {
      out->t = c.t;
      out->dt = c.dt;
      out->steps = c.steps;
    }
    out->inv_failures += (long long)c.counters[0];
    out->floor_hits += (long long)c.counters[1];
    out->unrecoverable += (long long)c.counters[2];
    unrec += c.counters[2];
    dterr += c.counters[3];
  }
  int rc = GRMHD_OK;
  if (check && unrec > dc->unrec_seen) rc = GRMHD_ERR_INVERSION;
  if (check && dterr > dc->dterr_seen) rc = GRMHD_ERR_DT;
  if (check) {
    dc->unrec_seen = unrec;
    dc->dterr_seen = dterr;
  }
  return rc;
}
