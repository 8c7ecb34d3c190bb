// elec_bodies.cuh -- the electron entropies of a grid (paper, "Implementation
// Notes": the optional partition of dissipation between ions and electrons
// of Ressler et al. 2015 with five heating models, and the bound P_gas /
// rho^gamma < 3 of the bounds list when electron temperatures are evolved).
//
// kappa_tot = P_gas/rho^gamma and kappa_e = P_e/rho^gamma_e ride with the
// mass.  Per stage, after the fluid's kernels:
//   elec_recon_body<d> reconstructs both entropies at the two faces of every
//                      zone along d (as recon_body does the primitives);
//   elec_flux_body<d>  (after the face fluxes of every direction) forms their
//                      local Lax-Friedrichs flux from the weights that the
//                      face kernels (FP64, FP32 or float-float) stored;
//   fix_flux_body      zeroes them where the mass flux is zeroed;
//   elec_post_body     (after the update, whose bounds wait for it) carries
//                      the entropies to the new state, heats the electrons by
//                      the model's share of the dissipation, applies the
//                      fluid's bounds (either frame), the entropy bound, the
//                      kappa_tot reset and the T_p/T_e bounds;
//   elec_fix_body      (after the fixup) gives a fixed-up zone the neighbour
//                      mean of kappa_e and the same closing steps.
#pragma once

#include "step_bodies.cuh"

namespace grmhd {

constexpr double KTOT_MAX = 3.0;          // P_gas / rho^gamma < 3
constexpr double ELEC_CLAMP = 1.0e20;     // T_p/T_e and beta_p within [1/C, C]
constexpr double MP_OVER_ME = 1836.15267343;
constexpr int FF_KTOT = 256;              // bound flag: u lowered for kappa_tot <= 3

// Powers of the density come from one logarithm per density value,
// rho^a = exp(a ln rho) (relative error about |a ln rho| x 1e-16, far below
// the step's rounding), instead of one pow() each.

// Heating share f_e of a zone (rho, u, kappa_e, b^2; lr = ln rho); models as
// documented with GRMHD_ELEC_* in grmhd.h.
static __device__ __noinline__ double elec_fraction(const StepArgs &A, double rho, double lr,
                                                    double u, double kel, double bsq) {
  if (A.elec == GRMHD_ELEC_CONSTANT) return A.fel_const;
  const double ue = kel * exp(A.game * lr) / (A.game - 1.0);
  const double Te = fabs((A.game - 1.0) * ue / rho);
  const double Tp = fabs((A.gamp - 1.0) * (u - ue) / rho);
  double trat = (Te > 0.0) ? Tp / Te : ELEC_CLAMP;  // T_p / T_e
  trat = fmin(fmax(trat, 1.0 / ELEC_CLAMP), ELEC_CLAMP);
  double beta = (bsq > 0.0) ? 2.0 * rho * Tp / bsq : ELEC_CLAMP;
  beta = fmin(fmax(beta, 1.0 / ELEC_CLAMP), ELEC_CLAMP);
  switch (A.elec) {
    case GRMHD_ELEC_KAWAZURA: {
      const double qiqe = 35.0 / (1.0 + pow(beta / 15.0, -1.4) * exp(-0.1 / trat));
      return 1.0 / (1.0 + qiqe);
    }
    case GRMHD_ELEC_WERNER: {
      const double s = bsq / rho;
      return 0.25 * (1.0 + sqrt((s / 5.0) / (2.0 + s / 5.0)));
    }
    case GRMHD_ELEC_ROWAN: {
      const double sw = bsq / (rho + A.gam * u);
      const double r = fmin(4.0 * sw * beta, 1.0);  // beta_p / beta_max
      return 0.5 * exp(-pow(1.0 - r, 3.3) / (1.0 + 1.2 * pow(sw, 0.7)));
    }
    case GRMHD_ELEC_SHARMA: {
      const double qeqi = 0.33 * sqrt(1.0 / trat);
      return qeqi / (1.0 + qeqi);
    }
    case GRMHD_ELEC_HOWES: {
      const double lt = log10(trat);
      const double c2 = (trat > 1.0) ? 1.6 / trat : 1.2 / trat;
      const double c3 = (trat > 1.0) ? 18.0 + 5.0 * lt : 18.0;
      const double bx = pow(beta, 2.0 - 0.2 * lt);
      const double qiqe = 0.92 * (c2 * c2 + bx) / (c3 * c3 + bx) * sqrt(MP_OVER_ME * trat) *
                          exp(-1.0 / beta);
      return 1.0 / (1.0 + qiqe);
    }
  }
  return 0.0;
}

// The closing steps of a zone once the fluid's bounds are done: u lowered
// to P_gas/rho^gamma = 3 where it exceeds that (with the bounds on),
// kappa_tot reset to (gamma - 1) u / rho^gamma, kappa_e held to
// tpte_min <= T_p/T_e <= tpte_max, i.e. within kappa_tot rho^(gamma -
// gamma_e) / ((gamma - 1)/(gamma_e - 1) + R (gamma - 1)/(gamma_p - 1)) at
// R = tpte_max .. tpte_min (a kappa_e that is not a number takes the lower).
// lr = ln P[RHO].
__device__ __forceinline__ int elec_close(const StepArgs &A, double P[NV], double K[2], double lr) {
  int fl = 0;
  const double g1 = A.gam - 1.0;
  const double rg = exp(A.gam * lr);
  if (A.floors_on) {
    const double kt = g1 * P[UU] / rg;
    if (kt > KTOT_MAX) {
      P[UU] = KTOT_MAX * rg / g1;
      fl = FF_KTOT;
    }
  }
  K[0] = g1 * P[UU] / rg;
  const double a = g1 / (A.game - 1.0), b = g1 / (A.gamp - 1.0);
  const double kk = K[0] * exp((A.gam - A.game) * lr);
  const double kmax = kk / (a + A.tpte_min * b);
  const double kmin = kk / (a + A.tpte_max * b);
  double kel = K[1];
  if (!(kel == kel)) kel = kmin;
  K[1] = fmin(fmax(kel, kmin), kmax);
  return fl;
}

// Zone-centric reconstruction of both entropies along DIR (the zones of
// recon_body): KLf = value at the zone's low face, KRf = at its high face,
// [2][ntot] each.
template <int DIR>
__device__ __forceinline__ void elec_recon_body(const StepArgs &A, const double *__restrict__ K,
                                                double *__restrict__ KLf,
                                                double *__restrict__ KRf, long long t) {
  const Dims &D = A.D;
  const int e0 = D.n[0] + 2, e1 = D.n[1] + 2;
  if (t >= n_recon(D, A.flat3)) return;
  const int i = NG - 1 + (int)(t % e0);
  const int j = NG - 1 + (int)((t / e0) % e1);
  const int k = (A.flat3 ? NG : NG - 1) + (int)(t / ((long long)e0 * e1));
  const long long c = zid(D, i, j, k);
  const long long st = (DIR == 0) ? 1 : (DIR == 1) ? D.s[0] : D.n2d;
#pragma unroll
  for (int q = 0; q < 2; q++) {
    const double *p = K + q * D.ntot + c;
    double lo, hi;
    if (A.recon == 1) {
      weno5_pair(__ldg(p - 2 * st), __ldg(p - st), __ldg(p), __ldg(p + st), __ldg(p + 2 * st), lo, hi);
    } else {
      const double x1 = __ldg(p), h = 0.5 * mc_slope(__ldg(p - st), x1, __ldg(p + st));
      lo = x1 - h;
      hi = x1 + h;
    }
    KLf[q * D.ntot + c] = lo;
    KRf[q * D.ntot + c] = hi;
  }
}

// Entropy fluxes of one face along DIR (the face box of face_body):
// F_K = w_L K_L + w_R K_R with K_L the high-face value of zone c-1, K_R the
// low-face value of zone c, and the weights the face kernel of the grid's
// precision stored, w_L = sqrt(-g)/2 rho_L (u^d_L + c u^t_L),
// w_R = sqrt(-g)/2 rho_R (u^d_R - c u^t_R) (c: the face's LLF speed), so
// that F_K is the LLF combination of rho u^d K and rho u^t K.
template <int DIR>
__device__ __forceinline__ void elec_flux_body(const StepArgs &A, const double *__restrict__ KLf,
                                               const double *__restrict__ KRf,
                                               double *__restrict__ FK, long long t) {
  const Dims &D = A.D;
  int lo[3], ext[3];
  face_box(D, DIR, A.flat3, lo, ext);
  if (t >= (long long)ext[0] * ext[1] * ext[2]) return;
  const int i = lo[0] + (int)(t % ext[0]);
  const int j = lo[1] + (int)((t / ext[0]) % ext[1]);
  const int k = lo[2] + (int)(t / ((long long)ext[0] * ext[1]));
  const long long c = zid(D, i, j, k), N = D.ntot;
  const long long st = (DIR == 0) ? 1 : (DIR == 1) ? D.s[0] : D.n2d;
  const double wl = A.elec_w[(2 * DIR) * N + c], wr = A.elec_w[(2 * DIR + 1) * N + c];
#pragma unroll
  for (int q = 0; q < 2; q++) FK[q * N + c] = wl * KRf[q * N + c - st] + wr * KLf[q * N + c];
}

// After the update: the entropies carried to the new state, U_K = U_rho(P_i)
// K_i - dt' div F_K and kappa_adv = U_K / U_rho(new), U_rho(new) = U_rho(P_i)
// - dt' div F_rho; then, in a zone whose inversion succeeded (Pout holds its
// unbounded state), the heating kappa_e = kappa_e,adv + f_e (gamma_e - 1) /
// (gamma - 1) rho_s^(gamma - gamma_e) ((gamma - 1) u/rho^gamma -
// kappa_tot,adv) with f_e from the source state P_s, the fluid's bounds and
// the closing steps.  U_rho(P_i) is formed in the predictor (P_i = P^n is
// intact there) and kept in Uek for the corrector, whose output overwrote
// P^n.  Every thread of the block must call it (warp counters).
__device__ __forceinline__ void elec_post_body(const StepArgs &A, const double *Ps, double *Pout,
                                               const double *__restrict__ F1,
                                               const double *__restrict__ F2,
                                               const double *__restrict__ F3,
                                               const double *__restrict__ FK1,
                                               const double *__restrict__ FK2,
                                               const double *__restrict__ FK3, const double *Ki,
                                               const double *Ks, double *Kout, double *Uek,
                                               const int *__restrict__ pflag, int *fflag,
                                               double dtfac, int stage, long long t) {
  const Dims &D = A.D;
  const double dt = A.clk->dt;
  if (!(dt > 0.0)) return;
  const double dtp = dtfac * dt;
  const bool active = t < n_zone(D);
  int ff = 0;
  if (active) {
    const int i = NG + (int)(t % D.n[0]);
    const int j = NG + (int)((t / D.n[0]) % D.n[1]);
    const int k = NG + (int)(t / ((long long)D.n[0] * D.n[1]));
    const long long c = zid(D, i, j, k), N = D.ntot;
    const long long ij = (long long)j * D.s[0] + i;
    Geo G;
    load_geo(A.geom, D.n2d, ij, G);
    double ps[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) ps[v] = Ps[v * N + c];
    FState ss;
    fluid_state(ps, G, ss);
    double Uri;
    if (stage == 0) {  // P_s = P_i = P^n
      Uri = G.gdet * (ps[RHO] * ss.ucon[0]);
      Uek[c] = Uri;
    } else {
      Uri = Uek[c];
    }
    const double idx1 = A.idx[0], idx2 = A.idx[1], idx3 = A.idx[2];
    const long long o = RHO * N + c;
    const double divr = (F1[o + 1] - F1[o]) * idx1 + (F2[o + D.s[0]] - F2[o]) * idx2 +
                        (F3[o + D.n2d] - F3[o]) * idx3;
    const double Urn = Uri + dtp * (0.0 - divr);
    double kn[2];
#pragma unroll
    for (int q = 0; q < 2; q++) {
      const long long oq = q * N + c;
      const double divk = (FK1[oq + 1] - FK1[oq]) * idx1 + (FK2[oq + D.s[0]] - FK2[oq]) * idx2 +
                          (FK3[oq + D.n2d] - FK3[oq]) * idx3;
      kn[q] = (Uri * Ki[oq] + dtp * (0.0 - divk)) / Urn;
    }
    if (pflag[c] == 0) {
      double pn[NV];
#pragma unroll
      for (int v = 0; v < NV; v++) pn[v] = Pout[v * N + c];
      const double ls = log(ps[RHO]), ln = log(pn[RHO]);
      const double fel = elec_fraction(A, ps[RHO], ls, ps[UU], Ks[N + c], ss.bsq);
      const double ktot_new = (A.gam - 1.0) * pn[UU] / exp(A.gam * ln);
      kn[1] = kn[1] + fel * (A.game - 1.0) / (A.gam - 1.0) * exp((A.gam - A.game) * ls) *
                          (ktot_new - kn[0]);
      const double rho_n = pn[RHO];
      if (A.floors_on) {
        const double rho_fl = __ldg(A.floors + ij), u_fl = __ldg(A.floors + D.n2d + ij);
        ff = A.floor_drift ? apply_floors_drift(pn, G, rho_fl, u_fl, A.gk)
                           : apply_floors(pn, G, rho_fl, u_fl, A.gk);
      }
      ff |= elec_close(A, pn, kn, (pn[RHO] == rho_n) ? ln : log(pn[RHO]));
#pragma unroll
      for (int v = 0; v < NV; v++) Pout[v * N + c] = pn[v];
      fflag[c] = ff;
    }
    Kout[c] = kn[0];
    Kout[N + c] = kn[1];
  }
  count_warp(active && ff != 0, &A.clk->counters[1]);
}

// After the fixup: a fixed-up zone takes the mean kappa_e of the same
// neighbours and the closing steps (its bound flags gain FF_KTOT where u
// was lowered).  Every thread of the block must call it (warp counters).
__device__ __forceinline__ void elec_fix_body(const StepArgs &A, double *P, double *K,
                                              const int *__restrict__ pflag, int *fflag,
                                              long long t) {
  const Dims &D = A.D;
  if (!(A.clk->dt > 0.0)) return;
  const bool active = t < n_zone(D);
  bool hit = false;
  if (active) {
    const int i = NG + (int)(t % D.n[0]);
    const int j = NG + (int)((t / D.n[0]) % D.n[1]);
    const int k = NG + (int)(t / ((long long)D.n[0] * D.n[1]));
    const long long c = zid(D, i, j, k), N = D.ntot;
    if (pflag[c] != 0) {
      double sum = 0.0;
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
            sum += K[N + nb];
            cnt++;
          }
      if (cnt > 0) {
        double p[NV], kn[2] = {0.0, sum / (double)cnt};
#pragma unroll
        for (int v = 0; v < NV; v++) p[v] = P[v * N + c];
        const int f = elec_close(A, p, kn, log(p[RHO]));
        P[UU * N + c] = p[UU];
        K[c] = kn[0];
        K[N + c] = kn[1];
        if (f) {
          hit = fflag[c] == 0;
          fflag[c] |= f;
        }
      }
    }
  }
  count_warp(hit, &A.clk->counters[1]);
}

}  // namespace grmhd
