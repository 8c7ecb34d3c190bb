// plan.cu -- the plan kernels of the predictor-corrector step and their
// enqueue functions (plan.h).  Each kernel maps its block to a grid through
// the class's block table and runs the per-thread body of that grid.
#include <cstring>
#include <vector>

#include "../../include/grmhd.h"
#include "grmhd_impl.h"
#include "mixed_bodies.cuh"
#include "plan.h"
#include "step_bodies.cuh"

namespace grmhd {

namespace {

struct BView {
  const StageItem *__restrict__ items;
  const int *__restrict__ map;  // grid of each block of this class
  const int *__restrict__ off;  // first block of each grid in this class
};

__device__ __forceinline__ int block_grid(const BView &V) { return __ldg(V.map + blockIdx.x); }
__device__ __forceinline__ long long block_tid(const BView &V, int g) {
  return (long long)((int)blockIdx.x - __ldg(V.off + g)) * BS + threadIdx.x;
}
// the stage arrays: 0 = P, 1 = Ph
__device__ __forceinline__ double *arr(const StageItem &it, int which) { return which ? it.Ph : it.P; }

template <int X>
__global__ void kp_bounds(BView V, int which) {
  const int g = block_grid(V);
  const StageItem &it = V.items[g];
  const long long t = block_tid(V, g);
  double *P = arr(it, which);
  if (X == 0) bounds_x1_body(it.A, P, t);
  if (X == 1) bounds_x2_body(it.A, P, t);
  if (X == 2) bounds_x3_body(it.A, P, t);
}

template <int DIR>
__global__ void __launch_bounds__(BS) kp_recon(BView V, int in) {
  const int g = block_grid(V);
  const StageItem &it = V.items[g];
  const long long t = block_tid(V, g);
  const double *Ps = arr(it, in);
  if (it.A.recon == 1)
    recon_body<DIR, 1>(it.A, Ps, it.Lf, it.Rf, t);
  else
    recon_body<DIR, 0>(it.A, Ps, it.Lf, it.Rf, t);
}

template <int DIR>
__global__ void __launch_bounds__(BS) kp_face(BView V, int in) {
  const int g = block_grid(V);
  const StageItem &it = V.items[g];
  const long long t = block_tid(V, g);
  const double *Lf = it.Lf, *Rf = it.Rf;
  if (DIR == 2 && it.A.flat3) Lf = Rf = arr(it, in);  // flat X3: the primitives
  face_body<DIR>(it.A, Lf, Rf, it.F[DIR], t);
}

__global__ void kp_to_f32(BView V, int in) {
  const int g = block_grid(V);
  const StageItem &it = V.items[g];
  to_f32_body(arr(it, in), it.Pf, (long long)NV * it.A.D.ntot, block_tid(V, g));
}

template <int DIR>
__global__ void __launch_bounds__(BS) kp_recon_f32(BView V) {
  const int g = block_grid(V);
  const StageItem &it = V.items[g];
  const long long t = block_tid(V, g);
  float *Lf = (float *)it.Lf, *Rf = (float *)it.Rf;
  if (it.A.recon == 1)
    recon_f32_body<DIR, 1>(it.A, it.Pf, Lf, Rf, t);
  else
    recon_f32_body<DIR, 0>(it.A, it.Pf, Lf, Rf, t);
}

template <int DIR>
__global__ void __launch_bounds__(BS) kp_face_f32(BView V) {
  const int g = block_grid(V);
  const StageItem &it = V.items[g];
  const long long t = block_tid(V, g);
  const float *Lf = (const float *)it.Lf, *Rf = (const float *)it.Rf;
  if (DIR == 2 && it.A.flat3) Lf = Rf = it.Pf;
  face_f32_body<DIR>(it.A, it.geomf, Lf, Rf, it.F[DIR], t);
}

__global__ void kp_replicate(BView V) {
  const int g = block_grid(V);
  const StageItem &it = V.items[g];
  replicate_body(it.A, it.F[0], it.F[1], it.F[2], block_tid(V, g));
}

__global__ void kp_fix(BView V) {
  const int g = block_grid(V);
  const StageItem &it = V.items[g];
  fix_flux_body(it.A, it.F[0], it.F[1], block_tid(V, g));
}

__global__ void kp_emf(BView V) {
  const int g = block_grid(V);
  const StageItem &it = V.items[g];
  emf_body(it.A, it.F[0], it.F[1], it.F[2], it.emf, block_tid(V, g));
}

__global__ void kp_ct(BView V) {
  const int g = block_grid(V);
  const StageItem &it = V.items[g];
  ct_body(it.A, it.F[0], it.F[1], it.F[2], it.emf, block_tid(V, g));
}

__global__ void __launch_bounds__(BS) kp_update(BView V, int in, double dtfac, int ucache_mode) {
  const int g = block_grid(V);
  const StageItem &it = V.items[g];
  update_body(it.A, it.P, arr(it, in), arr(it, 1 - in), it.F[0], it.F[1], it.F[2], it.pflag,
              it.fflag, dtfac, it.Uc, ucache_mode, block_tid(V, g));
}

__global__ void kp_fixup(BView V, int out) {
  const int g = block_grid(V);
  const StageItem &it = V.items[g];
  fixup_body(it.A, arr(it, out), it.pflag, it.fflag, block_tid(V, g));
}

// one thread per grid
__global__ void kp_clock(const StageItem *__restrict__ items, int ngrid, int op) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ngrid) return;
  const StageItem &it = items[g];
  if (op == 0) reset_ctop_body(it.A.clk);
  if (op == 1) dt_body(it.A);
  if (op == 2) advance_body(it.A);
}

long long nblk(long long n) { return (n + BS - 1) / BS; }

BView view(const Plan &p, int cls) {
  BView V;
  V.items = p.items;
  V.off = p.tab + p.off_base[cls];
  V.map = p.tab + p.map_base[cls];
  return V;
}

// Launch one kernel of class cls (skipped when no grid has blocks in it),
// bracketed for the hook as kernel class kclass.
template <typename L>
int launch(const Plan &p, int cls, int kclass, PlanHook *h, L &&body) {
  if (p.nblocks[cls] <= 0) return 0;
  if (h) h->begin(kclass, 1);
  body((unsigned)p.nblocks[cls], view(p, cls));
  if (h) h->end(kclass);
  return 1;
}

}  // namespace

int plan_build(Plan &p, const StageItem *items, int n) {
  memset(&p, 0, sizeof(p));
  if (!items || n < 1) return GRMHD_ERR_INVALID;
  long long tot[PC_N] = {0};
  std::vector<std::vector<int>> nb(PC_N, std::vector<int>(n));
  long long zones = 0;
  for (int g = 0; g < n; g++) {
    const Dims &D = items[g].A.D;
    const int fl = items[g].A.flat3, mx = items[g].mixed;
    long long c[PC_N];
    c[PC_BX1] = n_bounds_x1(D);
    c[PC_BX2] = n_bounds_x2(D);
    c[PC_BX3] = n_bounds_x3(D);
    c[PC_RECON01] = mx ? 0 : n_recon(D, fl);
    c[PC_RECON2] = (mx || fl) ? 0 : n_recon(D, 0);
    for (int d = 0; d < 3; d++) {
      c[PC_FACE0 + d] = mx ? 0 : n_face(D, d, fl);
      c[PC_FACE0F + d] = mx ? n_face(D, d, fl) : 0;
    }
    c[PC_TOF32] = mx ? (long long)NV * D.ntot : 0;
    c[PC_RECON01F] = mx ? n_recon(D, fl) : 0;
    c[PC_RECON2F] = (mx && !fl) ? n_recon(D, 0) : 0;
    c[PC_REPL] = fl ? n_replicate(D) : 0;
    c[PC_FIX] = n_fix(D);
    c[PC_EDGE] = n_edge(D);
    c[PC_ZONE] = n_zone(D);
    for (int q = 0; q < PC_N; q++) {
      nb[q][g] = (int)nblk(c[q]);
      tot[q] += nb[q][g];
      if (tot[q] >= (1ll << 31) - 1) return GRMHD_ERR_INVALID;
    }
    zones += n_zone(D);
  }
  std::vector<int> host;
  for (int q = 0; q < PC_N; q++) {
    p.nblocks[q] = (int)tot[q];
    p.off_base[q] = (int)host.size();
    int acc = 0;
    for (int g = 0; g < n; g++) {
      host.push_back(acc);
      acc += nb[q][g];
    }
    host.push_back(acc);
    p.map_base[q] = (int)host.size();
    for (int g = 0; g < n; g++) host.insert(host.end(), (size_t)nb[q][g], g);
  }
  if (cudaMalloc(&p.items, sizeof(StageItem) * n) != cudaSuccess ||
      cudaMalloc(&p.tab, sizeof(int) * host.size()) != cudaSuccess) {
    cudaGetLastError();
    plan_free(p);
    return GRMHD_ERR_NOMEM;
  }
  if (cudaMemcpy(p.items, items, sizeof(StageItem) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p.tab, host.data(), sizeof(int) * host.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess) {
    plan_free(p);
    return GRMHD_ERR_CUDA;
  }
  p.ngrid = n;
  p.zones = zones;
  return GRMHD_OK;
}

void plan_free(Plan &p) {
  if (p.items) cudaFree(p.items);
  if (p.tab) cudaFree(p.tab);
  p.items = nullptr;
  p.tab = nullptr;
  p.ngrid = 0;
}

int plan_clock(const Plan &p, int op, cudaStream_t st, PlanHook *h) {
  const int kc = (op == 1) ? GRMHD_K_DT : GRMHD_K_OTHER;
  if (h) h->begin(kc, 1);
  kp_clock<<<(unsigned)nblk(p.ngrid), BS, 0, st>>>(p.items, p.ngrid, op);
  if (h) h->end(kc);
  return 1;
}

int plan_fluxes(const Plan &p, int in, cudaStream_t st, PlanHook *h) {
  int nl = plan_clock(p, 0, st, h);
  const int R = GRMHD_K_RECON, F = GRMHD_K_FLUX;
  // FP64 grids
  nl += launch(p, PC_RECON01, R, h, [&](unsigned nb, BView V) { kp_recon<0><<<nb, BS, 0, st>>>(V, in); });
  nl += launch(p, PC_FACE0, F, h, [&](unsigned nb, BView V) { kp_face<0><<<nb, BS, 0, st>>>(V, in); });
  nl += launch(p, PC_RECON01, R, h, [&](unsigned nb, BView V) { kp_recon<1><<<nb, BS, 0, st>>>(V, in); });
  nl += launch(p, PC_FACE1, F, h, [&](unsigned nb, BView V) { kp_face<1><<<nb, BS, 0, st>>>(V, in); });
  nl += launch(p, PC_RECON2, R, h, [&](unsigned nb, BView V) { kp_recon<2><<<nb, BS, 0, st>>>(V, in); });
  nl += launch(p, PC_FACE2, F, h, [&](unsigned nb, BView V) { kp_face<2><<<nb, BS, 0, st>>>(V, in); });
  // mixed-precision grids
  nl += launch(p, PC_TOF32, R, h, [&](unsigned nb, BView V) { kp_to_f32<<<nb, BS, 0, st>>>(V, in); });
  nl += launch(p, PC_RECON01F, R, h, [&](unsigned nb, BView V) { kp_recon_f32<0><<<nb, BS, 0, st>>>(V); });
  nl += launch(p, PC_FACE0F, F, h, [&](unsigned nb, BView V) { kp_face_f32<0><<<nb, BS, 0, st>>>(V); });
  nl += launch(p, PC_RECON01F, R, h, [&](unsigned nb, BView V) { kp_recon_f32<1><<<nb, BS, 0, st>>>(V); });
  nl += launch(p, PC_FACE1F, F, h, [&](unsigned nb, BView V) { kp_face_f32<1><<<nb, BS, 0, st>>>(V); });
  nl += launch(p, PC_RECON2F, R, h, [&](unsigned nb, BView V) { kp_recon_f32<2><<<nb, BS, 0, st>>>(V); });
  nl += launch(p, PC_FACE2F, F, h, [&](unsigned nb, BView V) { kp_face_f32<2><<<nb, BS, 0, st>>>(V); });
  // flat-X3 grids
  nl += launch(p, PC_REPL, GRMHD_K_OTHER, h,
               [&](unsigned nb, BView V) { kp_replicate<<<nb, BS, 0, st>>>(V); });
  return nl;
}

int plan_fix_ct(const Plan &p, cudaStream_t st, PlanHook *h) {
  const int C = GRMHD_K_CT;
  int nl = launch(p, PC_FIX, C, h, [&](unsigned nb, BView V) { kp_fix<<<nb, BS, 0, st>>>(V); });
  nl += launch(p, PC_EDGE, C, h, [&](unsigned nb, BView V) { kp_emf<<<nb, BS, 0, st>>>(V); });
  nl += launch(p, PC_EDGE, C, h, [&](unsigned nb, BView V) { kp_ct<<<nb, BS, 0, st>>>(V); });
  return nl;
}

int plan_update(const Plan &p, int in, double dtfac, int ucache_mode, cudaStream_t st, PlanHook *h) {
  int nl = launch(p, PC_ZONE, GRMHD_K_UPDATE, h, [&](unsigned nb, BView V) {
    kp_update<<<nb, BS, 0, st>>>(V, in, dtfac, ucache_mode);
  });
  nl += launch(p, PC_ZONE, GRMHD_K_FIXUP, h,
               [&](unsigned nb, BView V) { kp_fixup<<<nb, BS, 0, st>>>(V, 1 - in); });
  return nl;
}

int plan_bounds(const Plan &p, int which, cudaStream_t st, PlanHook *h) {
  const int B = GRMHD_K_BOUNDS;
  int nl = launch(p, PC_BX1, B, h, [&](unsigned nb, BView V) { kp_bounds<0><<<nb, BS, 0, st>>>(V, which); });
  nl += launch(p, PC_BX2, B, h, [&](unsigned nb, BView V) { kp_bounds<1><<<nb, BS, 0, st>>>(V, which); });
  nl += launch(p, PC_BX3, B, h, [&](unsigned nb, BView V) { kp_bounds<2><<<nb, BS, 0, st>>>(V, which); });
  return nl;
}

int plan_stage(const Plan &p, int stage, int ucache_mode, cudaStream_t st, PlanHook *h) {
  int nl = plan_fluxes(p, stage, st, h);
  if (stage == 0) nl += plan_clock(p, 1, st, h);
  nl += plan_fix_ct(p, st, h);
  nl += plan_update(p, stage, stage ? 1.0 : 0.5, ucache_mode, st, h);
  nl += plan_bounds(p, 1 - stage, st, h);
  return nl;
}

int plan_steps(const Plan &p, int nsteps, cudaStream_t st, PlanHook *h) {
  int nl = 0;
  for (int n = 0; n < nsteps; n++) {
    nl += plan_stage(p, 0, 1, st, h);  // predictor keeps U(P^n)
    nl += plan_stage(p, 1, 2, st, h);  // corrector reads it back
    nl += plan_clock(p, 2, st, h);
  }
  return nl;
}

}  // namespace grmhd
