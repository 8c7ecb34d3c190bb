// step_bodies.cuh -- the per-thread bodies of the kernels of one
// predictor-corrector stage of the HARM scheme (iharm3D, arXiv:2110.10191):
//   bounds (ghost fill) -> zone-centric reconstruction -> face fluxes (LLF,
//   with a warp/block max of the signal speed for the CFL step) -> dt ->
//   boundary flux fixes -> flux-CT EMFs (Toth 2000; paper, "Implementation
//   Notes", first paragraph) -> update + 1D_W inversion + bounds (same
//   section) -> fixup of failed zones.
//
// Each body takes the step arguments of one grid and the linear index t of
// its thread within that grid's launch range.  The plan kernels (plan.cu)
// run them for one grid or many (t from the block's index within its grid);
// the allocation-free flux entry point's kernels (step.cu) for one.  A block
// never spans two grids: the block reductions (signal speed maxima, warp
// counts) see the threads of one grid only.
//
// Every thread owns one face, edge or zone; fields are SoA float64 in HBM
// with i fastest, so warps read and write 256-byte contiguous runs.
//
// Flat X3 (A.flat3: n3 = 1 with periodic X3): every k layer of the
// primitives is an exact copy of the single interior layer, so the fluxes
// along X1 and X2 are computed on that layer only and copied to the layers
// above and below it (replicate_body), and the X3 faces read the primitives
// themselves as their face states (reconstruction of constant data returns
// the data exactly).  The results are bitwise those of the full extent.
#pragma once

#include "grmhd_dev.cuh"
#include "grmhd_impl.h"

namespace grmhd {

constexpr int BS = 128;      // default threads per block of the stage kernels
constexpr int BS_MAX = 256;  // largest block the plan kernels are compiled for

__device__ __forceinline__ int wrap(int g, int n) {  // periodic image of ghost index g
  int q = (g - NG) % n;
  if (q < 0) q += n;
  return NG + q;
}

// ---------------------------------------------------------------------------
// Launch extents (threads per grid) of each body
// ---------------------------------------------------------------------------
__host__ __device__ inline long long n_bounds_x1(const Dims &D) {
  return (long long)D.n[1] * D.n[2] * 2 * NG;
}
__host__ __device__ inline long long n_bounds_x2(const Dims &D) {
  return (long long)D.s[0] * D.n[2] * 2 * NG;
}
__host__ __device__ inline long long n_bounds_x3(const Dims &D) { return D.n2d * 2 * NG; }
// zones whose two face values are reconstructed along one direction
__host__ __device__ inline long long n_recon(const Dims &D, int flat3) {
  return (long long)(D.n[0] + 2) * (D.n[1] + 2) * (flat3 ? 1 : D.n[2] + 2);
}
// longest FP64 reconstruction walk (zones per thread)
constexpr int RWALK = 16;
static_assert(RWALK <= 16, "weno5_walk unrolls over at most 16 zones");
// threads of the FP64 reconstruction along dir: one per column and segment
// of rw zones along dir (rw >= 2), or one per zone (rw = 1)
__host__ __device__ inline long long n_recon_walk(const Dims &D, int dir, int flat3, int rw) {
  const long long e[3] = {D.n[0] + 2, D.n[1] + 2, flat3 ? 1 : D.n[2] + 2};
  if (rw <= 1) return e[0] * e[1] * e[2];
  return e[0] * e[1] * e[2] / e[dir] * ((e[dir] + rw - 1) / rw);
}
// faces along dir: dir index NG .. n+NG, transverse NG-1 .. n+NG (flux-CT
// needs one transverse layer on each side); flat X3 keeps the k = NG layer
__host__ __device__ inline void face_box(const Dims &D, int dir, int flat3, int lo[3], int ext[3]) {
  for (int e = 0; e < 3; e++) {
    lo[e] = (e == dir) ? NG : NG - 1;
    ext[e] = (e == dir) ? D.n[e] + 1 : D.n[e] + 2;
  }
  if (flat3) {
    lo[2] = NG;
    ext[2] = 1;
  }
}
__host__ __device__ inline long long n_face(const Dims &D, int dir, int flat3) {
  int lo[3], ext[3];
  face_box(D, dir, flat3, lo, ext);
  return (long long)ext[0] * ext[1] * ext[2];
}
__host__ __device__ inline long long n_replicate(const Dims &D) { return D.n2d * NV; }
__host__ __device__ inline long long n_fix(const Dims &D) {
  return (long long)((D.n[0] > D.n[1]) ? D.n[0] + 2 : D.n[1] + 2) * (D.n[2] + 2);
}
__host__ __device__ inline long long n_edge(const Dims &D) {
  return (long long)(D.n[0] + 1) * (D.n[1] + 1) * (D.n[2] + 1);
}
__host__ __device__ inline long long n_zone(const Dims &D) {
  return (long long)D.n[0] * D.n[1] * D.n[2];
}

// ---------------------------------------------------------------------------
// Boundary conditions
// ---------------------------------------------------------------------------
// K (null without electrons): the two electron entropies, copied as scalars
__device__ __forceinline__ void copy_zone(const Dims &D, double *P, double *K, long long dst,
                                          long long src) {
#pragma unroll
  for (int v = 0; v < NV; v++) P[v * D.ntot + dst] = P[v * D.ntot + src];
  if (K) {
    K[dst] = K[src];
    K[D.ntot + dst] = K[D.ntot + src];
  }
}

// X1 ghosts for interior (j, k); one thread per (ghost layer, side, j, k)
__device__ __forceinline__ void bounds_x1_body(const StepArgs &A, double *P, double *K,
                                               long long t) {
  const Dims &D = A.D;
  if (t >= n_bounds_x1(D)) return;
  const int g = (int)(t % NG);
  const int side = (int)((t / NG) % 2);
  const long long r = t / (2 * NG);
  const int j = NG + (int)(r % D.n[1]);
  const int k = NG + (int)(r / D.n[1]);
  const int bc = A.bc[0][side];
  const int ig = side ? D.n[0] + NG + g : g;
  const long long d = zid(D, ig, j, k);
  if (bc == 0) {
    copy_zone(D, P, K, d, zid(D, wrap(ig, D.n[0]), j, k));
  } else if (bc == 1) {
    const int ia = side ? D.n[0] + NG - 1 : NG;
    copy_zone(D, P, K, d, zid(D, ia, j, k));
    const double *gd = A.geom + (LOC_CENT * G_NCOMP + G_GDET) * D.n2d;
    const double rs = gd[(long long)j * D.s[0] + ia] / gd[(long long)j * D.s[0] + ig];
    P[B1 * D.ntot + d] *= rs;
    P[B2 * D.ntot + d] *= rs;
    P[B3 * D.ntot + d] *= rs;
    const double u1 = P[U1 * D.ntot + d];
    if (side == 0 ? (u1 > 0.0) : (u1 < 0.0)) P[U1 * D.ntot + d] = 0.0;
  }
}

// X2 ghosts for all i and interior k
__device__ __forceinline__ void bounds_x2_body(const StepArgs &A, double *P, double *K,
                                               long long t) {
  const Dims &D = A.D;
  if (t >= n_bounds_x2(D)) return;
  const int i = (int)(t % D.s[0]);
  const long long r = t / D.s[0];
  const int g = (int)(r % NG);
  const int side = (int)((r / NG) % 2);
  const int k = NG + (int)(r / (2 * NG));
  const int bc = A.bc[1][side];
  const int jg = side ? D.n[1] + NG + g : NG - 1 - g;
  const long long d = zid(D, i, jg, k);
  if (bc == 0) {
    copy_zone(D, P, K, d, zid(D, i, wrap(jg, D.n[1]), k));
  } else if (bc == 2) {
    const int jm = side ? D.n[1] + NG - 1 - g : NG + g;
    copy_zone(D, P, K, d, zid(D, i, jm, k));
    P[U2 * D.ntot + d] = -P[U2 * D.ntot + d];
    P[B2 * D.ntot + d] = -P[B2 * D.ntot + d];
  } else if (bc == 1) {
    copy_zone(D, P, K, d, zid(D, i, side ? D.n[1] + NG - 1 : NG, k));
  }
}

// X3 ghosts for all i, j
__device__ __forceinline__ void bounds_x3_body(const StepArgs &A, double *P, double *K,
                                               long long t) {
  const Dims &D = A.D;
  const long long nrow = D.n2d;
  if (t >= n_bounds_x3(D)) return;
  const long long ij = t % nrow;
  const long long r = t / nrow;
  const int g = (int)(r % NG);
  const int side = (int)(r / NG);
  const int bc = A.bc[2][side];
  const int kg = side ? D.n[2] + NG + g : NG - 1 - g;
  const long long d = (long long)kg * D.n2d + ij;
  if (bc == 0) {
    copy_zone(D, P, K, d, (long long)wrap(kg, D.n[2]) * D.n2d + ij);
  } else if (bc == 1) {
    copy_zone(D, P, K, d, (long long)(side ? D.n[2] + NG - 1 : NG) * D.n2d + ij);
  }
}

// ---------------------------------------------------------------------------
// Face fluxes
// ---------------------------------------------------------------------------
// Block maximum of v >= 0 (any block size that is a multiple of 32, up to
// 1024), one atomicMax per block; every thread of the block must call it.
__device__ __forceinline__ void warp_block_max(double v, unsigned long long *dst) {
  // v >= 0: its bit pattern orders like the value
  unsigned long long b = __double_as_longlong(v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long x = __shfl_xor_sync(0xffffffffu, b, o);
    b = (x > b) ? x : b;
  }
  __shared__ unsigned long long sm[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sm[w] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    unsigned long long m = sm[0];
    for (int q = 1; q < nw; q++) m = (sm[q] > m) ? sm[q] : m;
    if (m) atomicMax(dst, m);
  }
}

// Zone-centric reconstruction: both face values of each zone's 8 primitives
// along DIR (zones NG-1 .. n+NG along DIR and the extended transverse
// range), each zone's WENO smoothness indicators formed once.  With
// A.rwalk >= 2 one thread walks a segment of A.rwalk zones of one column
// along DIR, so consecutive zones share their differences (weno5_walk);
// consecutive threads take neighbouring columns (along X2 for DIR = 0, along
// X1 otherwise).  With A.rwalk = 1 (grids too small to fill the GPU with
// walks) one thread takes one zone, consecutive threads along X1.  Same
// values either way.  Lf = value at the zone's low face, Rf = at its high
// face.
template <int DIR, int RECON>
__device__ __forceinline__ void recon_body(const StepArgs &A, const double *__restrict__ P,
                                           double *__restrict__ Lf, double *__restrict__ Rf,
                                           long long t) {
  const Dims &D = A.D;
  const int e0 = D.n[0] + 2, e1 = D.n[1] + 2, e2 = A.flat3 ? 1 : D.n[2] + 2;
  const int kb = A.flat3 ? NG : NG - 1;
  const long long st = (DIR == 0) ? 1 : (DIR == 1) ? D.s[0] : D.n2d;
  const int rw = A.rwalk;
  if (rw <= 1) {
    if (t >= (long long)e0 * e1 * e2) return;
    const long long c = zid(D, NG - 1 + (int)(t % e0), NG - 1 + (int)((t / e0) % e1),
                            kb + (int)(t / ((long long)e0 * e1)));
#pragma unroll
    for (int v = 0; v < NV; v++) {
      const double *p = P + v * D.ntot + c;
      double lo, hi;
      if (RECON == 1) {
        weno5_pair(__ldg(p - 2 * st), __ldg(p - st), __ldg(p), __ldg(p + st), __ldg(p + 2 * st),
                   lo, hi);
      } else {
        const double x1 = __ldg(p), h = 0.5 * mc_slope(__ldg(p - st), x1, __ldg(p + st));
        lo = x1 - h;
        hi = x1 + h;
      }
      Lf[v * D.ntot + c] = lo;
      Rf[v * D.ntot + c] = hi;
    }
    return;
  }
  const int ed = (DIR == 0) ? e0 : (DIR == 1) ? e1 : e2;
  const int ea = (DIR == 0) ? e1 : e0;  // the column index that varies fastest
  const int eb = (DIR == 2) ? e1 : e2;
  const int nseg = (ed + rw - 1) / rw;
  if (t >= (long long)ea * eb * nseg) return;
  const int ca = (int)(t % ea);
  const long long r = t / ea;
  const int cb = (int)(r % eb);
  const int m0 = (int)(r / eb) * rw;
  const int i = NG - 1 + ((DIR == 0) ? m0 : ca);
  const int j = NG - 1 + ((DIR == 1) ? m0 : (DIR == 0) ? ca : cb);
  const int k = (DIR == 2) ? NG - 1 + m0 : kb + cb;
  const int n = min(rw, ed - m0);
  const long long c = zid(D, i, j, k);
#pragma unroll 1
  for (int v = 0; v < NV; v++) {
    const double *p = P + v * D.ntot + c;
    double *lf = Lf + v * D.ntot + c, *rf = Rf + v * D.ntot + c;
    if (RECON == 1) {
      weno5_walk(p, lf, rf, st, n);
    } else {
      for (int m = 0; m < n; m++) {
        const double *q = p + m * st;
        const double x1 = __ldg(q), h = 0.5 * mc_slope(__ldg(q - st), x1, __ldg(q + st));
        lf[m * st] = x1 - h;
        rf[m * st] = x1 + h;
      }
    }
  }
}

// The WENO5 reconstruction along X1 with each warp's rows staged in shared
// memory.  The lanes of a warp walk 32 different rows (neighbouring j), so
// their direct loads and stores touch 32 rows' sectors per instruction; here
// the warp loads its rows' stencil values together (consecutive addresses),
// walks them in shared memory, collects the face values of 8 zones per row
// and writes them back row by row.  Same arithmetic and results as
// recon_body<0, 1>, for A.rwalk >= 2.  Every thread of the block must call it
// (warp synchronisation); wsm: the warp's X1_WARP_BYTES of shared memory.
constexpr int X1_IN = RWALK + 5;  // a row's values at zones -2 .. RWALK+1, odd stride
constexpr int X1_OUT = 9;         // 8 face values per row and chunk, odd stride
constexpr int X1_HI = 32 * X1_OUT + 8;  // offset of the high-face chunk (another bank half)
constexpr int X1_WARP_BYTES = (32 * X1_IN + 2 * X1_HI) * 8 + 32 * 8 + 32 * 4;

__device__ __forceinline__ void recon_x1_staged(const StepArgs &A, const double *__restrict__ P,
                                                double *__restrict__ Lf, double *__restrict__ Rf,
                                                long long t, unsigned char *wsm) {
  const Dims &D = A.D;
  const int e0 = D.n[0] + 2, e1 = D.n[1] + 2, e2 = A.flat3 ? 1 : D.n[2] + 2;
  const int rw = A.rwalk;  // 2 .. RWALK
  const int nseg = (e0 + rw - 1) / rw;
  const int lane = threadIdx.x & 31;
  double *tin = reinterpret_cast<double *>(wsm);
  double *tout = tin + 32 * X1_IN;
  long long *rbase = reinterpret_cast<long long *>(tout + 2 * X1_HI);
  int *rn = reinterpret_cast<int *>(rbase + 32);
  int n = 0;  // this lane's zones (0: past the end of the grid's threads)
  long long c = 0;
  if (t < (long long)e1 * e2 * nseg) {
    const int ca = (int)(t % e1);
    const long long r = t / e1;
    const int cb = (int)(r % e2);
    const int m0 = (int)(r / e2) * rw;
    c = zid(D, NG - 1 + m0, NG - 1 + ca, (A.flat3 ? NG : NG - 1) + cb);
    n = min(rw, e0 - m0);
  }
  rbase[lane] = c;
  rn[lane] = n;
  if (n == 0)  // a row past the end is never loaded: its walk reads zeros, stores nothing
    for (int q = 0; q < X1_IN; q++) tin[lane * X1_IN + q] = 0.0;
  __syncwarp();
  const double *x = tin + lane * X1_IN;  // x[q]: this row's value at zone q - 2
#pragma unroll 1
  for (int v = 0; v < NV; v++) {
    const long long ov = v * D.ntot;
#pragma unroll 4
    for (int e = lane; e < 32 * (RWALK + 4); e += 32) {
      const int q = e / (RWALK + 4), xq = e - q * (RWALK + 4);
      const int nq = rn[q];  // rows past the end (nq = 0) load nothing
      if (nq > 0 && xq < nq + 4) tin[q * X1_IN + xq] = __ldg(P + ov + rbase[q] - 2 + xq);
    }
    __syncwarp();
    const double xm1 = x[1];
    double x0 = x[2], xp1 = x[3], xp2 = x[4];
    double dm1 = x0 - xm1, dp1 = xp1 - x0, dp2 = xp2 - xp1;
    double D0 = dm1 - (xm1 - x[0]), D1 = dp1 - dm1, D2 = dp2 - dp1;
    double T0 = weno5_T(D0), T1 = weno5_T(D1), T2 = weno5_T(D2);
#pragma unroll
    for (int m = 0; m < RWALK; m++) {
      if (m < n) {
        double lo, hi;
        weno5_pair_dt(x0, dm1, dp1, D0, D1, D2, T0, T1, T2, lo, hi);
        tout[lane * X1_OUT + (m & 7)] = lo;
        tout[X1_HI + lane * X1_OUT + (m & 7)] = hi;
        if (m + 1 < n) {
          const double dn = x[m + 5] - xp2;
          x0 = xp1;
          xp1 = xp2;
          xp2 = x[m + 5];
          dm1 = dp1;
          dp1 = dp2;
          D0 = D1;
          D1 = D2;
          D2 = dn - dp2;
          dp2 = dn;
          T0 = T1;
          T1 = T2;
          T2 = weno5_T(D2);
        }
      }
      if ((m & 7) == 7) {  // write zones m-7 .. m of every row: 4 rows x 8 zones per store
        __syncwarp();
#pragma unroll
        for (int it = 0; it < 16; it++) {
          const int e = it * 32 + lane;
          const int q = (e >> 3) & 31, col = e & 7, z = (m & ~7) + col;
          if (z < rn[q]) {
            double *dst = (it < 8) ? Lf : Rf;
            dst[ov + rbase[q] + z] = tout[((it < 8) ? 0 : X1_HI) + q * X1_OUT + col];
          }
        }
        __syncwarp();
      }
    }
  }
}

// One thread per face combines Rf of zone c-1 (left state) and Lf of zone c
// (right state) into the LLF flux; every thread of the block must call it.
// ELEC: the grid evolves electron entropies, whose flux weights it stores.
template <int DIR, bool ELEC = false>
__device__ __forceinline__ void face_body(const StepArgs &A, const double *__restrict__ Lf,
                                          const double *__restrict__ Rf, double *__restrict__ F,
                                          long long t) {
  const Dims &D = A.D;
  int lo[3], ext[3];
  face_box(D, DIR, A.flat3, lo, ext);
  const long long nface = (long long)ext[0] * ext[1] * ext[2];
  const bool active = t < nface;
  double ctop = 0.0;
  if (active) {
    const int i = lo[0] + (int)(t % ext[0]);
    const int j = lo[1] + (int)((t / ext[0]) % ext[1]);
    const int k = lo[2] + (int)(t / ((long long)ext[0] * ext[1]));
    const long long c = zid(D, i, j, k);
    const long long st = (DIR == 0) ? 1 : (DIR == 1) ? D.s[0] : D.n2d;
    double PL[NV], PR[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) {
      PL[v] = __ldg(Rf + v * D.ntot + c - st);
      PR[v] = __ldg(Lf + v * D.ntot + c);
    }
    const int loc = (DIR == 0) ? LOC_FACE1 : (DIR == 1) ? LOC_FACE2 : LOC_CENT;
    Geo G;
    load_geo(A.geom + (long long)loc * G_NCOMP * D.n2d, D.n2d, (long long)j * D.s[0] + i, G);
    FState sL, sR;
    fluid_state(PL, G, sL);
    fluid_state(PR, G, sR);
    // c_top = max(0, vmax_L, vmax_R, -vmin_L, -vmin_R): the larger root
    // magnitude of either side
    const double ct = fmax(mhd_cmax(PL, sL, G, A.gam, A.ggm1, DIR + 1),
                           mhd_cmax(PR, sR, G, A.gam, A.ggm1, DIR + 1));
    // LLF: F = 1/2 sqrt(-g) [(F_L + ct U_L) + (F_R - ct U_R)]
    double acc[NV];
    flux_cons_acc<true>(PL, sL, A.gm1, DIR + 1, ct, acc);
    const double mL = acc[RHO];  // rho_L (u^d_L + ct u^t_L): the left mass term
    flux_cons_acc<false>(PR, sR, A.gm1, DIR + 1, -ct, acc);
    const double hg = 0.5 * G.gdet;
#pragma unroll
    for (int v = 0; v < NV; v++) F[v * D.ntot + c] = hg * acc[v];
    if (ELEC) {  // the electron entropies' flux weights (LLF of rho u^d K, rho u^t K)
      A.elec_w[(2 * DIR) * D.ntot + c] = hg * mL;
      A.elec_w[(2 * DIR + 1) * D.ntot + c] = hg * (acc[RHO] - mL);
    }
    bool interior = true;
#pragma unroll
    for (int e = 0; e < 3; e++) {
      if (e == DIR) continue;
      const int q = (e == 0) ? i : (e == 1) ? j : k;
      interior = interior && (q >= NG) && (q < D.n[e] + NG);
    }
    if (interior) ctop = ct;
  }
  warp_block_max(ctop, &A.clk->ctop_bits[DIR]);
}

// Flat X3: copy the k = NG layer of F1 and F2 to k = NG-1 and NG+1, and of
// F3 to k = NG+1 (one thread per (variable, i, j)).
__device__ __forceinline__ void replicate_body(const StepArgs &A, double *F1, double *F2, double *F3,
                                               long long t) {
  const Dims &D = A.D;
  if (t >= n_replicate(D)) return;
  const long long v = t / D.n2d, ij = t % D.n2d;
  const long long c = v * D.ntot + NG * D.n2d + ij;
  const double f1 = F1[c], f2 = F2[c], f3 = F3[c];
  F1[c - D.n2d] = f1;
  F1[c + D.n2d] = f1;
  F2[c - D.n2d] = f2;
  F2[c + D.n2d] = f2;
  F3[c + D.n2d] = f3;
}

__device__ __forceinline__ void reset_ctop_body(Clock *clk) {
  clk->ctop_bits[0] = clk->ctop_bits[1] = clk->ctop_bits[2] = 0ull;
}

// ---------------------------------------------------------------------------
// Time step: ndt_d = cfl dx_d / max ctop_d over directions with n_d > 1,
// dt = 1/sum(1/ndt_d), dt <= 1.3 dt_prev, last step lands on t_final.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void dt_body(const StepArgs &A) {
  Clock *c = A.clk;
  double inv = 0.0;
  for (int d = 0; d < 3; d++) {
    if (A.D.n[d] <= 1) continue;
    const double ct = __longlong_as_double((long long)c->ctop_bits[d]);
    if (ct > 0.0) {
      const double ndt = __ddiv_rn(A.cfl * A.dx[d], ct);
      inv = __dadd_rn(inv, __ddiv_rn(1.0, ndt));
    }
  }
  double dt = (inv > 0.0) ? __ddiv_rn(1.0, inv) : __longlong_as_double(0x7ff0000000000000ll);
  if (c->dt_prev > 0.0 && dt > 1.3 * c->dt_prev) dt = 1.3 * c->dt_prev;
  if (c->t_final > 0.0 && __dadd_rn(c->t, dt) > c->t_final) dt = __dadd_rn(c->t_final, -c->t);
  if (!isfinite(dt)) {  // every signal speed zero: no CFL step exists
    c->counters[3] += 1;
    dt = 0.0;
  }
  if (!(dt > 0.0)) dt = 0.0;
  c->dt = dt;
}

__device__ __forceinline__ void advance_body(const StepArgs &A) {
  Clock *c = A.clk;
  if (c->dt > 0.0 && isfinite(c->dt)) {
    c->t = __dadd_rn(c->t, c->dt);
    c->dt_prev = c->dt;
    c->steps += 1;
  }
}

// ---------------------------------------------------------------------------
// Boundary flux fixes and flux-CT
// ---------------------------------------------------------------------------
// FK1, FK2 (null without electrons): the electron entropy fluxes of X1 and
// X2 faces, zeroed with the polar fluxes and with a zeroed mass inflow.
__device__ __forceinline__ void fix_flux_body(const StepArgs &A, double *F1, double *F2,
                                              double *FK1, double *FK2, long long t) {
  const Dims &D = A.D;
  // polar faces: (i, k) over the extended ranges
  const long long np = (long long)(D.n[0] + 2) * (D.n[2] + 2);
  const long long nr = (long long)(D.n[1] + 2) * (D.n[2] + 2);
  if (t < np) {
    const int i = NG - 1 + (int)(t % (D.n[0] + 2));
    const int k = NG - 1 + (int)(t / (D.n[0] + 2));
    if (A.bc[1][0] == 2) {
      const long long c = zid(D, i, NG, k);
      for (int v = 0; v < NV; v++) F2[v * D.ntot + c] = 0.0;
      if (FK2) FK2[c] = FK2[D.ntot + c] = 0.0;
    }
    if (A.bc[1][1] == 2) {
      const long long c = zid(D, i, D.n[1] + NG, k);
      for (int v = 0; v < NV; v++) F2[v * D.ntot + c] = 0.0;
      if (FK2) FK2[c] = FK2[D.ntot + c] = 0.0;
    }
  }
  if (t < nr) {
    const int j = NG - 1 + (int)(t % (D.n[1] + 2));
    const int k = NG - 1 + (int)(t / (D.n[1] + 2));
    if (A.bc[0][0] == 1) {
      const long long c = zid(D, NG, j, k);
      double *f = F1 + RHO * D.ntot + c;
      if (*f > 0.0) {
        *f = 0.0;
        if (FK1) FK1[c] = FK1[D.ntot + c] = 0.0;
      }
    }
    if (A.bc[0][1] == 1) {
      const long long c = zid(D, D.n[0] + NG, j, k);
      double *f = F1 + RHO * D.ntot + c;
      if (*f < 0.0) {
        *f = 0.0;
        if (FK1) FK1[c] = FK1[D.ntot + c] = 0.0;
      }
    }
  }
}

// Edge EMFs over i, j, k in [NG, n+NG]:
// e3 = (F1[B2] + F1[B2](j-1) - F2[B1] - F2[B1](i-1))/4, cyclic for e1, e2.
__device__ __forceinline__ void emf_body(const StepArgs &A, const double *__restrict__ F1,
                                         const double *__restrict__ F2,
                                         const double *__restrict__ F3, double *__restrict__ emf,
                                         long long t) {
  const Dims &D = A.D;
  const int e0 = D.n[0] + 1, e1 = D.n[1] + 1;
  if (t >= n_edge(D)) return;
  const int i = NG + (int)(t % e0);
  const int j = NG + (int)((t / e0) % e1);
  const int k = NG + (int)(t / ((long long)e0 * e1));
  const long long c = zid(D, i, j, k), N = D.ntot;
  const long long im = c - 1, jm = c - D.s[0], km = c - D.n2d;
  emf[2 * N + c] = 0.25 * (F1[B2 * N + c] + F1[B2 * N + jm] - F2[B1 * N + c] - F2[B1 * N + im]);
  emf[1 * N + c] = 0.25 * (F3[B1 * N + c] + F3[B1 * N + im] - F1[B3 * N + c] - F1[B3 * N + km]);
  emf[0 * N + c] = 0.25 * (F2[B3 * N + c] + F2[B3 * N + km] - F3[B2 * N + c] - F3[B2 * N + jm]);
}

// Induction fluxes from the EMFs on every face the update reads.
__device__ __forceinline__ void ct_body(const StepArgs &A, double *F1, double *F2, double *F3,
                                        const double *__restrict__ emf, long long t) {
  const Dims &D = A.D;
  const int e0 = D.n[0] + 1, e1 = D.n[1] + 1;
  if (t >= n_edge(D)) return;
  const int i = NG + (int)(t % e0);
  const int j = NG + (int)((t / e0) % e1);
  const int k = NG + (int)(t / ((long long)e0 * e1));
  const long long c = zid(D, i, j, k), N = D.ntot;
  const double *E1 = emf, *E2 = emf + N, *E3 = emf + 2 * N;
  const bool in1 = i < D.n[0] + NG, in2 = j < D.n[1] + NG, in3 = k < D.n[2] + NG;
  if (in2 && in3) {  // X1 face
    F1[B1 * N + c] = 0.0;
    F1[B2 * N + c] = 0.5 * (E3[c] + E3[c + D.s[0]]);
    F1[B3 * N + c] = -0.5 * (E2[c] + E2[c + D.n2d]);
  }
  if (in1 && in3) {  // X2 face
    F2[B1 * N + c] = -0.5 * (E3[c] + E3[c + 1]);
    F2[B2 * N + c] = 0.0;
    F2[B3 * N + c] = 0.5 * (E1[c] + E1[c + D.n2d]);
  }
  if (in1 && in2) {  // X3 face
    F3[B1 * N + c] = 0.5 * (E2[c] + E2[c + 1]);
    F3[B2 * N + c] = -0.5 * (E1[c] + E1[c + D.s[0]]);
    F3[B3 * N + c] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// Update + inversion + floors, one thread per interior zone.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void count_warp(bool pred, unsigned long long *ctr) {
  const unsigned m = __ballot_sync(0xffffffffu, pred);
  if (m && (threadIdx.x & 31) == 0) atomicAdd(ctr, (unsigned long long)__popc(m));
}

__device__ __forceinline__ void geo_source(const double P[NV], const FState &s, const Geo &G,
                                           const double *__restrict__ conn, long long n2d,
                                           long long ij, double gam, double S[4]) {
  // S_nu = sqrt(-g) T^k_l Gamma^l_{nu k}
  const double pg = (gam - 1.0) * P[UU];
  const double w = P[RHO] + P[UU] + pg + s.bsq;
  const double pt = pg + 0.5 * s.bsq;
  double T[4][4];
#pragma unroll
  for (int m = 0; m < 4; m++) {
#pragma unroll
    for (int n = 0; n < 4; n++) T[m][n] = w * s.ucon[m] * s.ucov[n] - s.bcon[m] * s.bcov[n];
    T[m][m] += pt;
  }
#pragma unroll
  for (int nu = 0; nu < 4; nu++) {
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
      for (int l = 0; l < 4; l++) acc += T[k][l] * __ldg(conn + (l * 10 + SY(nu, k)) * n2d + ij);
    S[nu] = acc * G.gdet;
  }
}

// Ucache: the predictor stores U(P^n) there and the corrector, whose P_i is
// the same P^n, reads it back instead of recomputing it (null: neither).
// Every thread of the block must call it (warp counters).
__device__ __forceinline__ void update_body(const StepArgs &A, const double *Pi,
                                            const double *__restrict__ Ps, double *Pout,
                                            const double *__restrict__ F1,
                                            const double *__restrict__ F2,
                                            const double *__restrict__ F3, int *pflag, int *fflag,
                                            double dtfac, double *Ucache, int ucache_mode,
                                            long long t) {
  const Dims &D = A.D;
  const double dt = A.clk->dt;
  if (!(dt > 0.0)) return;  // uniform across the grid: no warp divergence
  const double dtp = dtfac * dt;
  const long long nz = n_zone(D);
  const bool active = t < nz;
  int pf = 0, ff = 0;
  if (active) {
    const int i = NG + (int)(t % D.n[0]);
    const int j = NG + (int)((t / D.n[0]) % D.n[1]);
    const int k = NG + (int)(t / ((long long)D.n[0] * D.n[1]));
    const long long c = zid(D, i, j, k), N = D.ntot;
    const long long ij = (long long)j * D.s[0] + i;
    Geo G;
    load_geo(A.geom, D.n2d, ij, G);
    double pi[NV], ps[NV], Ui[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) pi[v] = Pi[v * N + c];
    double S[4];
    if (Ps == Pi) {
      FState si;
      fluid_state(pi, G, si);
      prim_flux(pi, si, G, A.gam, 0, Ui);
      if (ucache_mode == 1) {
#pragma unroll
        for (int v = 0; v < NV; v++) Ucache[v * N + c] = Ui[v];
      }
      geo_source(pi, si, G, A.conn, D.n2d, ij, A.gam, S);
    } else {
      if (ucache_mode == 2) {
#pragma unroll
        for (int v = 0; v < NV; v++) Ui[v] = Ucache[v * N + c];
      } else {
        FState si;
        fluid_state(pi, G, si);
        prim_flux(pi, si, G, A.gam, 0, Ui);
      }
#pragma unroll
      for (int v = 0; v < NV; v++) ps[v] = Ps[v * N + c];
      FState ss;
      fluid_state(ps, G, ss);
      geo_source(ps, ss, G, A.conn, D.n2d, ij, A.gam, S);
    }
    const double idx1 = A.idx[0], idx2 = A.idx[1], idx3 = A.idx[2];
    double Un[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) {
      const long long o = v * N + c;
      const double div = (F1[o + 1] - F1[o]) * idx1 + (F2[o + D.s[0]] - F2[o]) * idx2 +
                         (F3[o + D.n2d] - F3[o]) * idx3;
      // the source enters the energy and momentum rows only
      Un[v] = (v >= UU && v <= U3) ? fma(dtp, S[v - UU] - div, Ui[v]) : fma(-dtp, div, Ui[v]);
    }
    double pn[NV], bsq_n = 0.0, lor_n = 1.0;
    pf = invert_1dw(Un, G, A.gk, pi, pn, bsq_n, lor_n);
    if (pf == PF_OK && A.floors_on && !A.floor_drift && !A.elec)
      ff = apply_floors_known(pn, G, __ldg(A.floors + ij), __ldg(A.floors + D.n2d + ij), A.gk,
                              bsq_n, lor_n);
#pragma unroll
    for (int v = 0; v < NV; v++) Pout[v * N + c] = pn[v];
    pflag[c] = pf;
    fflag[c] = ff;
  }
  count_warp(active && pf != 0, &A.clk->counters[0]);
  count_warp(active && ff != 0, &A.clk->counters[1]);
}

// ---------------------------------------------------------------------------
// Drift-frame bounds of the zones whose inversion succeeded (the update
// leaves their bounds to this pass when A.floor_drift is set).  Every thread
// of the block must call it (warp counters).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void floor_drift_body(const StepArgs &A, double *P,
                                                 const int *__restrict__ pflag, int *fflag,
                                                 long long t) {
  const Dims &D = A.D;
  if (!(A.clk->dt > 0.0)) return;
  const long long nz = n_zone(D);
  const bool active = t < nz;
  int ff = 0;
  if (active) {
    const int i = NG + (int)(t % D.n[0]);
    const int j = NG + (int)((t / D.n[0]) % D.n[1]);
    const int k = NG + (int)(t / ((long long)D.n[0] * D.n[1]));
    const long long c = zid(D, i, j, k), N = D.ntot;
    if (pflag[c] == 0) {
      const long long ij = (long long)j * D.s[0] + i;
      Geo G;
      load_geo(A.geom, D.n2d, ij, G);
      double p[NV];
#pragma unroll
      for (int v = 0; v < NV; v++) p[v] = P[v * N + c];
      ff = apply_floors_drift(p, G, __ldg(A.floors + ij), __ldg(A.floors + D.n2d + ij), A.gk);
      if (ff) {
#pragma unroll
        for (int v = 0; v < NV; v++) P[v * N + c] = p[v];
        fflag[c] = ff;
      }
    }
  }
  count_warp(active && ff != 0, &A.clk->counters[1]);
}

// ---------------------------------------------------------------------------
// Fixup: a failed zone takes the mean of rho, u, utilde over the non-failed
// interior zones of its 3x3x3 neighbourhood (B is kept), then the bounds.
// Every thread of the block must call it (warp counters).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void fixup_body(const StepArgs &A, double *P, const int *__restrict__ pflag,
                                           int *fflag, long long t) {
  const Dims &D = A.D;
  if (!(A.clk->dt > 0.0)) return;
  const long long nz = n_zone(D);
  const bool active = t < nz;
  bool hit = false, lost = false;
  if (active) {
    const int i = NG + (int)(t % D.n[0]);
    const int j = NG + (int)((t / D.n[0]) % D.n[1]);
    const int k = NG + (int)(t / ((long long)D.n[0] * D.n[1]));
    const long long c = zid(D, i, j, k), N = D.ntot;
    if (pflag[c] != 0) {
      double sum[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      int cnt = 0;
      for (int dk = -1; dk <= 1; dk++)
        for (int dj = -1; dj <= 1; dj++)
          for (int di = -1; di <= 1; di++) {
            if (di == 0 && dj == 0 && dk == 0) continue;
            const int ii = i + di, jj = j + dj, kk = k + dk;
            if (ii < NG - A.xlo[0] || ii >= D.n[0] + NG + A.xhi[0] || jj < NG - A.xlo[1] ||
                jj >= D.n[1] + NG + A.xhi[1] || kk < NG - A.xlo[2] || kk >= D.n[2] + NG + A.xhi[2])
              continue;
            const long long nb = zid(D, ii, jj, kk);
            if (pflag[nb] != 0) continue;
#pragma unroll
            for (int v = 0; v < 5; v++) sum[v] += P[v * N + nb];
            cnt++;
          }
      if (cnt == 0) {
        lost = true;
      } else {
        double p[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) p[v] = P[v * N + c];
#pragma unroll
        for (int v = 0; v < 5; v++) p[v] = sum[v] / (double)cnt;
        if (A.floors_on) {
          const long long ij = (long long)j * D.s[0] + i;
          Geo G;
          load_geo(A.geom, D.n2d, ij, G);
          const int f = apply_floors(p, G, __ldg(A.floors + ij), __ldg(A.floors + D.n2d + ij), A.gk);
          if (f) {
            fflag[c] |= f;
            hit = true;
          }
        }
#pragma unroll
        for (int v = 0; v < NV; v++) P[v * N + c] = p[v];
      }
    }
  }
  count_warp(hit, &A.clk->counters[1]);
  count_warp(lost, &A.clk->counters[2]);
}

}  // namespace grmhd
