/*
 * grmhd.h -- C ABI of the GB300 (sm_103a) GRMHD step library.
 *
 * The library advances the equations of ideal general-relativistic MHD on a
 * fixed, stationary metric with the HARM conservative finite-volume scheme
 * that iharm3D implements (arXiv:2110.10191, "Functionality and Purpose"):
 * a logically Cartesian mesh in arbitrary coordinates, primitives in,
 * primitives after N predictor-corrector steps out.  Each step is
 *   predictor: fluxes of P^n -> CFL time step -> U(P^n) + dt/2 (-div F + S)
 *              -> 1D_W inversion (paper, "Implementation Notes", third
 *              paragraph) -> bounds (same section, list of bounds) -> fixup;
 *   corrector: fluxes of P^{n+1/2} -> U(P^n) + dt (-div F + S) -> ... -> P^{n+1},
 * with flux-CT constrained transport (same section, first paragraph) and a
 * metric evaluated numerically from its analytic line element (second
 * paragraph).  Units GM = c = 1 (fourth paragraph).
 *
 * Conventions shared by every call:
 *   - Primitives P: 8 variables in the order rho, u (internal energy
 *     density), utilde^1..3 (4-velocity relative to the normal observer),
 *     B^1..3 (= *F^{it}).  Arrays are structure-of-arrays, float64,
 *     P[v][k][j][i] with i fastest.  "Interior" arrays are [8][n3][n2][n1];
 *     "ghost" arrays include 3 ghost layers per side:
 *     [8][n3+6][n2+6][n1+6].
 *   - on_device = 1: the pointer is a CUDA device pointer valid on the
 *     simulation's stream (e.g. a torch tensor's data_ptr()); 0: host memory
 *     (pageable or pinned).  Host copies are synchronous with respect to the
 *     caller; device copies are ordered on the stream.
 *   - Ownership: the library owns every device buffer of a simulation; the
 *     caller owns the buffers it passes.  Nothing is retained after a call.
 *   - Errors: every call returns GRMHD_OK (0) or a negative code; no call
 *     aborts, exits or throws.  grmhd_strerror() names a code.
 *   - All entry points are thread-compatible, not thread-safe: one
 *     simulation must not be used from two threads at once.
 */
#ifndef GRMHD_H
#define GRMHD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GRMHD_OK 0
#define GRMHD_ERR_INVALID (-1)   /* bad argument, size or enum */
#define GRMHD_ERR_NOMEM (-2)     /* device allocation failed */
#define GRMHD_ERR_CUDA (-3)      /* a CUDA runtime call failed */
#define GRMHD_ERR_INVERSION (-4) /* a failed zone had no valid neighbour */
#define GRMHD_ERR_DT (-5)        /* no finite time step (all signal speeds zero) */

#define GRMHD_METRIC_MINKOWSKI 0 /* Cartesian flat space */
#define GRMHD_METRIC_MKS_KERR 1  /* Kerr in modified Kerr-Schild coordinates */

#define GRMHD_BC_PERIODIC 0
#define GRMHD_BC_OUTFLOW 1 /* X1 only: copy, sqrt(-g) B constant, no inflow */
#define GRMHD_BC_POLAR 2   /* X2 only: reflect, utilde^2 and B^2 negated */
#define GRMHD_BC_FIXED 3   /* ghosts keep the values last set */

#define GRMHD_RECON_MC 0
#define GRMHD_RECON_WENO5 1

#define GRMHD_PREC_FP64 0  /* every step in FP64 */
#define GRMHD_PREC_MIXED 1 /* reconstruction, fluid states, signal speeds and LLF fluxes
                              in FP32; geometry, flux-CT, update, inversion, bounds FP64 */
#define GRMHD_PREC_FF 2    /* float-float: reconstruction, fluxes, U(P), geometric source
                              and the 1D_W inversion in pairs of FP32 words (~48
                              significant bits) on the FP32 pipe, in per-zone scaled
                              units; flux divergence, flux-CT, bounds and the state FP64 */
#define GRMHD_PREC_MIXED_FF 3 /* the fluxes of GRMHD_PREC_MIXED (FP32) with the update of
                                 GRMHD_PREC_FF (float-float U(P), source, inversion) */

typedef struct grmhd_sim grmhd_sim; /* opaque, library-owned */

/* Logically Cartesian mesh of n1 x n2 x n3 zones on [xmin, xmax] per
 * direction (code coordinates X^1..3).  n3 = 1 (and n2 = 1) give 2D (1D)
 * problems; every direction still carries 3 ghost layers. */
typedef struct {
  int n1, n2, n3;
  double x1min, x1max, x2min, x2max, x3min, x3max;
} grmhd_grid;

/* Stationary metric.  MKS: r = exp(X1), theta = pi X2 + (1-hslope)/2
 * sin(2 pi X2), phi = X3, Kerr of mass 1 and spin a in Kerr-Schild form. */
typedef struct {
  int kind;
  double a, hslope;
} grmhd_metric;

/* Electron thermodynamics (paper, "Implementation Notes": the optional
 * tracking and partition of dissipation between ions and electrons of
 * Ressler et al. 2015, with five heating models).  The total entropy
 * kappa_tot = P_gas/rho^gamma and the electron entropy kappa_e =
 * P_e/rho^gamma_e are carried with the mass (conserved sqrt(-g) rho u^t
 * kappa, fluxes from kappa reconstructed like the primitives and combined
 * by the same local Lax-Friedrichs rule).  After each stage's inversion the
 * dissipation kappa_tot(u) - kappa_tot,carried heats the electrons by the
 * share f_e of the chosen model, evaluated on the stage's source state:
 * kappa_e += f_e (gamma_e - 1)/(gamma - 1) rho_s^(gamma - gamma_e) x that
 * difference.  The fluid's bounds follow; then u is lowered to keep
 * P_gas/rho^gamma <= 3 (with the bounds on), kappa_tot is reset to the
 * state's and kappa_e is held to tpte_min <= T_p/T_e <= tpte_max.  A failed
 * zone takes the neighbour mean of kappa_e.  Every heating model: f_e =
 * 1/(1 + Q_i/Q_e), T_e, T_p from kappa_e and u, beta_p = rho T_p / (b^2/2),
 * T_p/T_e clamped to [1e-20, 1e20], beta_p to [1e-20, 1e20]:
 *   KAWAZURA  Q_i/Q_e = 35/(1 + (beta_p/15)^-1.4 exp(-0.1 T_e/T_p))
 *   WERNER    f_e = (1 + sqrt((s/5)/(2 + s/5)))/4, s = b^2/rho
 *   ROWAN     f_e = exp(-(1 - beta_p/beta_max)^3.3/(1 + 1.2 s_w^0.7))/2,
 *             s_w = b^2/(rho + u + p), beta_max = 1/(4 s_w), beta_p <= beta_max
 *   SHARMA    Q_e/Q_i = 0.33 sqrt(T_e/T_p)
 *   HOWES     Q_i/Q_e = 0.92 (c2^2 + beta_p^x)/(c3^2 + beta_p^x)
 *             sqrt(m_p T_p/(m_e T_e)) exp(-1/beta_p), x = 2 - 0.2 log10(T_p/T_e),
 *             c2 = 1.6 T_e/T_p, c3 = 18 + 5 log10(T_p/T_e) (T_p > T_e), else
 *             c2 = 1.2 T_e/T_p, c3 = 18
 *   CONSTANT  f_e = fel (not one of the paper's models; for tests)
 * Grids of every precision mode evolve them (the mass-flux weights of the
 * entropy fluxes come from the grid's face kernels, in their arithmetic;
 * everything else about the entropies is FP64); decomposed grids exchange
 * them with the primitives; server requests carry them
 * (grmhd_server_submit_electrons). */
#define GRMHD_ELEC_OFF 0
#define GRMHD_ELEC_CONSTANT 1
#define GRMHD_ELEC_KAWAZURA 2
#define GRMHD_ELEC_WERNER 3
#define GRMHD_ELEC_ROWAN 4
#define GRMHD_ELEC_SHARMA 5
#define GRMHD_ELEC_HOWES 6

typedef struct {
  int model;                  /* GRMHD_ELEC_*; 0 (zero-initialised): off */
  double game, gamp;          /* adiabatic indices of electrons and protons (> 1) */
  double fel;                 /* GRMHD_ELEC_CONSTANT's share, in [0, 1] */
  double tpte_min, tpte_max;  /* 0 <= tpte_min <= tpte_max (may be +inf) */
} grmhd_electrons;

/* gamma: adiabatic index; cfl: Courant number; t_final > 0 clamps the last
 * step to land on it (steps after it do nothing); recon: GRMHD_RECON_*;
 * floors_on: apply the paper's bounds (needs the MKS radius); bc[d][side]:
 * GRMHD_BC_* for direction d, side 0 = low, 1 = high; precision:
 * GRMHD_PREC_* (the state, geometry and conserved variables are FP64 in
 * every mode); floor_frame: GRMHD_FLOOR_* (0, the fluid frame, when
 * zero-initialised). */
typedef struct {
  double gamma, cfl, t_final;
  int recon, floors_on;
  int bc[3][2];
  int precision;
  int floor_frame; /* GRMHD_FLOOR_*: where the bounds add mass and energy */
  grmhd_electrons electrons; /* electron entropies (model 0: not evolved) */
} grmhd_params;

/* Frame of the bounds (the paper lists the bounds, not the frame in which
 * they add material).  FLUID: rho and u are raised in place, the velocity
 * is kept.  DRIFT: the same mass and internal energy are added as a
 * field-free parcel moving with the drift velocity (the normal-observer
 * 3-velocity minus its component along B), its conserved variables added to
 * U(P) and the sum inverted by 1D_W; the fluid-frame bounds then run once
 * more so that every bound holds.  The frames agree where the flow is
 * perpendicular to B, and where B is absent: g_ij B^i B^j <= 1e-20 rho.  Fixed-up zones take the fluid-frame bounds in
 * either frame. */
#define GRMHD_FLOOR_FLUID 0
#define GRMHD_FLOOR_DRIFT 1


/* Running statistics of a simulation (totals over all stages so far). */
typedef struct {
  double t, dt;                  /* current time, last step's dt */
  long long steps;               /* full steps taken */
  long long inv_failures;        /* zones whose 1D_W inversion failed */
  long long floor_hits;          /* zones in which any bound acted */
  long long unrecoverable;       /* failed zones with no valid neighbour */
} grmhd_stats;

/* Allocate a simulation on the current CUDA device and build its geometry
 * (metric, inverse, sqrt(-g), lapse at zone centres and faces, numerical
 * connection at centres).  The problem it states is the paper's
 * ("Functionality and Purpose": ideal GRMHD in a stationary spacetime on a
 * logically Cartesian mesh in arbitrary coordinates); the metric quantities
 * are evaluated numerically from the analytic line element ("Implementation
 * Notes", second paragraph).  stream: a cudaStream_t (NULL = legacy default
 * stream) on which every later call of this simulation is ordered.
 * n1, n2, n3 >= 1 and (n1+6)(n2+6)(n3+6) < 2^31.  *out is set on success. */
int grmhd_create(const grmhd_grid *grid, const grmhd_metric *metric,
                 const grmhd_params *params, void *stream, grmhd_sim **out);

/* Free every device buffer.  NULL is accepted.  (The end of the
 * simulation's lifetime; the paper has no separate passage for it.) */
int grmhd_destroy(grmhd_sim *sim);

/* Set the interior primitives ([8][n3][n2][n1]) and fill the ghosts by the
 * boundary conditions.  The primitive variables (density, internal energy,
 * velocity; "Implementation Notes", third paragraph) and the field are the
 * state the scheme evolves ("Functionality and Purpose"). */
int grmhd_set_prims(grmhd_sim *sim, const double *P, int on_device);

/* Set primitives including ghosts ([8][n3+6][n2+6][n1+6]); the boundary
 * conditions then refill every non-FIXED ghost region. */
int grmhd_set_prims_ghost(grmhd_sim *sim, const double *P, int on_device);

/* Read the primitives, interior ([8][n3][n2][n1]) or with ghosts: the
 * state after the steps taken, recovered from the conserved variables by
 * the 1D_W inversion and bounded ("Implementation Notes", third paragraph
 * and list of bounds). */
int grmhd_get_prims(grmhd_sim *sim, double *P, int with_ghosts, int on_device);

/* The electron entropies (kappa_tot, kappa_e) of a simulation created with
 * electrons: K is [2][n3][n2][n1] (with_ghosts = 0; the ghosts are then
 * filled by the boundary conditions, FIXED ghosts kept) or [2][n3+6][n2+6]
 * [n1+6] (with_ghosts = 1); set them after the primitives.
 * GRMHD_ERR_INVALID: no electrons. */
int grmhd_set_electrons(grmhd_sim *sim, const double *K, int with_ghosts, int on_device);
int grmhd_get_electrons(grmhd_sim *sim, double *K, int with_ghosts, int on_device);

/* Advance nsteps full predictor-corrector steps, enqueued on the stream:
 * the conservative HARM update ("Functionality and Purpose") with flux-CT
 * ("Implementation Notes", first paragraph), the 1D_W inversion (third
 * paragraph) and the bounds at the end of each stage (list of bounds); the
 * predictor-corrector, reconstruction, LLF fluxes and fixup are the HARM
 * method of Gammie et al. (2003), which the paper builds on and does not
 * print.
 * stats == NULL: returns after enqueueing (errors of this call surface at
 * the next synchronising call).  stats != NULL: synchronises, fills *stats
 * and returns GRMHD_ERR_INVERSION if any failed zone had no valid neighbour
 * since the previous synchronising call.  With nsteps >= 2 and profiling
 * off, the cycles are replays of a CUDA graph of one cycle (captured on the
 * first such call, on a stream of the simulation's own that is ordered
 * after and before the simulation's stream): the same kernels and results,
 * without a host launch per kernel. */
int grmhd_step(grmhd_sim *sim, int nsteps, grmhd_stats *stats);

/* Synchronise and read the running statistics. */
int grmhd_get_stats(grmhd_sim *sim, grmhd_stats *stats);

/* Restore the clock of a checkpoint: time t, the previous step's dt (the
 * next step's growth limit depends on it) and the step count. */
int grmhd_set_time(grmhd_sim *sim, double t, double dt_prev, long long steps);

/* ---- Stage-level access, for verification of the individual steps ---- */

/* Predictor stage only: P <- P^{n+1/2} (time and step count unchanged). */
int grmhd_predictor(grmhd_sim *sim);

/* Face fluxes of the current state after the boundary flux fixes and
 * flux-CT, into host memory F[3][8][n3+6][n2+6][n1+6] (face i-1/2 of zone
 * i stored at zone i; entries outside the computed face ranges are zero),
 * and the maximum signal speed over interior faces per direction ctop[3]. */
int grmhd_get_fluxes(grmhd_sim *sim, double *F, double *ctop);

/* The time step the next step would take (host value). */
int grmhd_next_dt(grmhd_sim *sim, double *dt);

/* Inversion failure code and bound flags of the last stage, interior
 * [n3][n2][n1] int32, into host memory. */
int grmhd_get_flags(grmhd_sim *sim, int *pflag, int *fflag);

/* Geometry at location loc (0 zone centre, 1 X1 face, 2 X2 face) as host
 * out[34][n2+6][n1+6]: g_{mu nu} (16, row-major), g^{mu nu} (16), sqrt(-g),
 * lapse; loc 3 gives the connection Gamma^l_{m n} out[64][n2+6][n1+6]
 * (index (l*4+m)*4+n) at zone centres. */
int grmhd_get_geometry(grmhd_sim *sim, int loc, double *out);

/* Replace the geometry at location loc with caller-supplied values, in the
 * spirit of the paper's numerically evaluated metric ("Implementation
 * Notes", second paragraph: any stationary spacetime whose metric is known
 * runs on the same scheme), in the layout grmhd_get_geometry() returns
 * (host memory; loc 0..2: g_{mu nu},
 * g^{mu nu}, sqrt(-g), lapse; loc 3: the connection).  Only the upper
 * triangle (m <= n) of each symmetric index pair is read.  This runs the
 * step on a tabulated metric (any stationary, X3-independent spacetime
 * whose line element the library does not build in) and lets a test hold
 * the geometry fixed while it checks the step.  The bound thresholds keep
 * following the built-in radius r = exp(X1). */
int grmhd_set_geometry(grmhd_sim *sim, int loc, const double *in);

/* Kernel classes of the step, for grmhd_get_profile(). */
#define GRMHD_K_FLUX 0    /* LLF face fluxes from reconstructed states (3 launches a stage;
                             in the FP32-flux modes with the reconstruction fused in) */
#define GRMHD_K_DT 1      /* CFL time step */
#define GRMHD_K_CT 2      /* boundary flux fixes + flux-CT */
#define GRMHD_K_UPDATE 3  /* conserved update + 1D_W inversion + bounds */
#define GRMHD_K_FIXUP 4   /* fixup of failed zones */
#define GRMHD_K_BOUNDS 5  /* ghost fill */
#define GRMHD_K_OTHER 6   /* clock advance, signal-speed reset */
#define GRMHD_K_RECON 7   /* MC / WENO5 reconstruction of face states (3 launches a stage;
                             in the FP32-flux modes the FP32 copy of the stage input) */
#define GRMHD_NKCLASS 8

typedef struct {
  double ms[GRMHD_NKCLASS];            /* summed device time per class */
  long long launches[GRMHD_NKCLASS];   /* kernels launched per class */
} grmhd_profile_data;

/* enable != 0: record CUDA events on the simulation's stream around each
 * kernel class of the following steps (timing); launches are always
 * counted.  The events add no synchronisation. */
int grmhd_profile(grmhd_sim *sim, int enable);

/* Synchronise and read the per-class device times and launch counts since
 * the last reset; reset != 0 clears them afterwards. */
int grmhd_get_profile(grmhd_sim *sim, grmhd_profile_data *out, int reset);

/* The flux-CT invariant of the current state: *divb_max = the largest
 * |corner-centred divergence of sqrt(-g) B| over the corners between
 * interior zones (sum over directions with more than one zone of the
 * difference of sqrt(-g) B^d between the 4 zones on either side of the
 * corner, over 4 dX_d), and *gb_max (may be NULL) = the largest
 * |sqrt(-g) B^d| of those zones; flux-CT keeps their ratio, times the
 * smallest dX, at round-off.  Synchronises the stream. */
int grmhd_divb(grmhd_sim *sim, double *divb_max, double *gb_max);

/* Autotuner: pick, by timing on the simulation's stream, the threads per
 * block (64, 128 or 256) of each heavy kernel of the step (reconstruction,
 * face fluxes, update + fixup, in the simulation's precision).  Results do
 * not depend on the choice: each thread computes the same zone or face
 * whatever the block size.  The trial launches write only scratch (face
 * values, fluxes, the interior of the half-step array) and the inversion
 * and bound flags of the last stage; the state and the clock are left as
 * they were.  Synchronises the device.  trials >= 1 timed passes per
 * candidate; *ms_before / *ms_after (either may be NULL): one pass of the
 * tuned kernels with the previous and the chosen settings. */
int grmhd_autotune(grmhd_sim *sim, int trials, double *ms_before, double *ms_after);

/* Zones per thread of the FP64 reconstruction ("Implementation Notes",
 * WENO5 / linear reconstruction).  With 2, 4, 8 or 16, one thread walks
 * that many consecutive zones of a column along the direction, and
 * consecutive zones share their stencil differences. With 1, one thread
 * takes one zone.  0 restores the automatic choice: the longest walk that
 * still gives every reconstruction launch 152 x 640 threads, else 1.  The
 * values do not depend on the setting; only the launch shape and the FP64
 * instruction count do.  Synchronises the device.  *chosen (may be NULL)
 * receives the length in use.  GRMHD_ERR_INVALID for other values. */
int grmhd_set_recon_walk(grmhd_sim *sim, int zones_per_thread, int *chosen);

/* Measured double-precision FMA throughput of the current device: runs a
 * dependency-free DFMA kernel for about `iters` FMAs per thread on every SM
 * and returns FLOP/s (2 per FMA) in *flops.  Used as the roofline peak of
 * the FP64-bound kernels. */
int grmhd_fp64_peak(long long iters, double *flops);

/* The FP64 issue rate of the current device: thread-level FP64 instructions
 * (op 0: fused multiply-add, 1: add, 2: multiply) per SM per SM clock
 * cycle, from a loop of `chains` (1, 2, 4, 8 or 16) independent dependent
 * chains per thread on blocks_per_sm (1..16) blocks of 128 threads per SM,
 * about `iters` iterations per thread; the SM clock (*sm_mhz) is measured
 * inside the kernel (SM cycle counter against the global nanosecond
 * timer) and the time by CUDA events.  The FP64-bound kernels of the step
 * are reported against the rate it finds. */
int grmhd_fp64_probe(int op, int chains, int blocks_per_sm, long long iters,
                     double *ops_per_sm_clock, double *sm_mhz);

/* The reciprocal, reciprocal square root and square root that the step
 * uses inside its arithmetic (WENO5 weights, fluid states, signal speeds,
 * the Newton iteration of the 1D_W inversion; the paper's "Implementation
 * Notes" name the inversion, the HARM method the rest), on n device doubles
 * x into out, enqueued on stream; for verification of the step's
 * arithmetic.  fn 0: 1/x, the hardware approximation refined by one
 * third-order step of the geometric series; fn 1: 1/sqrt(x), the hardware
 * approximation refined by the binomial series to second order; fn 2:
 * sqrt(x) = x times fn 1.  Each is within 2 ulp of the IEEE result for
 * normal x in [2^-1022, 2^1022] (positive for fn 1, 2).  Outside that range
 * the approximations flush subnormal inputs and results to zero: for fn 0 a
 * zero or subnormal x gives NaN and |x| > 2^1022 a zero of x's sign; the
 * step sends zero and subnormal arguments of fn 2 to a branch of its own.
 * fn 3, 4: the quotients of the bounds ("Implementation Notes", list of
 * bounds), x / 400 (b^2 / sigma_max) and x / 100 (u / T-bound), by one
 * correction step from the divisor's correctly rounded reciprocal: the IEEE
 * quotient bit for bit for finite x whose quotient is normal.
 * GRMHD_ERR_INVALID: fn outside 0..4, n < 0, NULL pointers with n > 0. */
int grmhd_arith(int fn, const double *x, double *out, long long n, void *stream);

/* Face-flux stage without any device allocation (no counterpart in the
 * paper: it exists for callers of this library that cannot allocate).
 * Serving processes that have reserved all device memory up front, code
 * running under a framework allocator that must not be bypassed, and host
 * threads that may not allocate while other work is in flight cannot call
 * cudaMalloc; this call lets them run the flux stage (reconstruction + LLF
 * fluxes, boundary flux fixes, flux-CT) of the step on buffers they own.
 *   P:    device, primitives with ghosts [8][n3+6][n2+6][n1+6], ghosts
 *         already filled (e.g. grmhd_get_prims(..., with_ghosts=1, ...)).
 *   F:    device, output [3][8][n3+6][n2+6][n1+6], as grmhd_get_fluxes
 *         fills it (entries outside the computed face ranges are zeroed).
 *   ctop: host double[3] for the interior signal-speed maxima, or NULL;
 *         when given, the call synchronises the stream to read them.
 * grid, metric and params are checked as grmhd_create checks them; the
 * fluxes are FP64 whatever params->precision says (fields the flux stage
 * does not read are ignored).
 * Every intermediate (metric at centres and faces, EMFs, signal-speed
 * maxima) lives in one file-scope device array of 64 MiB that every GPU
 * loading this library holds until exit.  A grid needs 24 N + 936 A bytes
 * of it plus at most 1 KiB of alignment, N = (n1+6)(n2+6)(n3+6) and
 * A = (n1+6)(n2+6) (3 EMFs per zone; 117 doubles of geometry, connection
 * and bound thresholds per (i, j)): cubes up to 123^3 fit, and a grid that
 * does not is refused with GRMHD_ERR_INVALID.  The call makes no
 * cudaMalloc, cudaFree or allocating library call.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current and keeps it (behind a lock: calls may come from
 * several threads); make that first call before any stream capture.  A
 * call that meets a CUDA error forgets the address, so that after a device
 * reset the next call looks it up again.  All calls share the array and it
 * keeps the last call's contents: calls that overlap on the GPU (other
 * streams, other threads) race on it and must be serialised. */
int grmhd_fluxes_noalloc(const grmhd_grid *grid, const grmhd_metric *metric,
                         const grmhd_params *params, const double *P, double *F,
                         double *ctop, void *stream);

/* ---- Batches: many independent grids advanced by one set of launches ----
 *
 * The paper scales by giving each node its own mesh block ("Scaling"
 * section) and tests that the evolution does not depend on how the domain
 * is split (end of its "Tests" section).  On one GPU, independent grids are
 * the units: one launch of each kernel of the stage covers every grid of a
 * batch, so small grids (2D problems, many served requests) do not leave
 * most SMs idle, and a step costs the same launches whatever the number of
 * grids (32 when every grid is FP64; mixed-precision grids add the FP32
 * flux kernels).  Each grid keeps its own buffers, geometry, boundary
 * conditions, reconstruction, precision, CFL time step and clock (t_final
 * included).  A simulation stepped alone runs the same kernels as a batch
 * of one, so a grid's state after n batched steps is bitwise its state
 * after grmhd_step(sim, n) alone. */
typedef struct grmhd_batch grmhd_batch; /* opaque, library-owned */

typedef struct {
  int ngrid;              /* grids in the batch */
  long long zones;        /* interior zones over all grids */
  int launches_per_step;  /* kernels launched per batched step (0 before the first) */
  long long launches;     /* kernels launched by grmhd_batch_step so far */
  int graph;              /* 1 once a CUDA graph of the step has been captured */
  int tuned;              /* 1 after grmhd_batch_autotune */
  int recon_walk;         /* zones per thread of the FP64 reconstruction (1: one per
                             zone; see grmhd_set_recon_walk), chosen over all grids */
} grmhd_batch_info;

/* Group nsims simulations (created by grmhd_create on the current device;
 * each at most once) into a batch.  The batch references them and owns
 * none: destroy the batch before any of its simulations.  It has its own
 * CUDA stream.  GRMHD_ERR_INVALID: a NULL or repeated simulation, or more
 * than 2^31 - 1 blocks in one launch. */
int grmhd_batch_create(grmhd_sim *const *sims, int nsims, grmhd_batch **out);

/* Free the batch (its simulations are untouched).  NULL is accepted. */
int grmhd_batch_destroy(grmhd_batch *batch);

/* Advance every grid nsteps predictor-corrector steps, asynchronously:
 * the batch's stream first waits for the work already enqueued on each
 * member's stream, and each member's stream then waits for the batch, so
 * calls on a member (grmhd_get_prims, grmhd_get_stats, grmhd_step) stay
 * ordered after it.  use_graph != 0: the first call captures one step into
 * a CUDA graph and every step replays it.  Per-grid statistics and the
 * unrecoverable-zone check: grmhd_get_stats / grmhd_step(sim, 0, &stats). */
int grmhd_batch_step(grmhd_batch *batch, int nsteps, int use_graph);

/* The autotuner of grmhd_autotune over the batch's launches: per heavy
 * kernel, the threads per block (64, 128, 256) and the order in which the
 * grids' blocks are issued (plan order; largest grid first; round robin
 * over the grids).  Results do not depend on either choice.  A captured
 * graph is dropped and captured again at the next graph step. */
int grmhd_batch_autotune(grmhd_batch *batch, int trials, double *ms_before, double *ms_after);

/* Block orders for grmhd_batch_set_launch. */
#define GRMHD_ORDER_GRID 0 /* grids in batch order, each grid's blocks together */
#define GRMHD_ORDER_LPT 1  /* grids by decreasing block count (largest first) */
#define GRMHD_ORDER_RR 2   /* round robin: one block of each grid in turn */

/* Set by hand what grmhd_batch_autotune picks, for the kernels of class
 * kclass (GRMHD_K_RECON, GRMHD_K_FLUX or GRMHD_K_UPDATE; the update's
 * class also sets the fixup): threads per block (64..256, a multiple of 32)
 * and block order (GRMHD_ORDER_*).  Results do not depend on either.
 * Synchronises the device; a captured graph is dropped. */
int grmhd_batch_set_launch(grmhd_batch *batch, int kclass, int threads, int order);

/* Size and launch counts of the batch. */
int grmhd_batch_get_info(grmhd_batch *batch, grmhd_batch_info *out);

/* Wait for the batch's stream. */
int grmhd_batch_sync(grmhd_batch *batch);

/* Device bytes grmhd_create would allocate for this grid (state, stage
 * scratch, fluxes, geometry, flags, clock, the FP32 copies of the mixed
 * mode and the launch plan); GRMHD_ERR_INVALID as grmhd_create. */
int grmhd_footprint(const grmhd_grid *grid, const grmhd_metric *metric,
                    const grmhd_params *params, size_t *bytes);

/* ---- Serving: a request loop over simulations that arrive over time ----
 *
 * No counterpart in the paper (it runs one simulation per job).  A server
 * owns a thread that takes submitted simulations in arrival order, admits
 * each when its device footprint fits the server's HBM budget (and, if
 * set, when the zones in flight stay under a cap), in arrival order or
 * smallest work first, keeps the admitted
 * states resident, and advances all of them together: each round is one
 * batch step (grmhd_batch_*) of up to `quantum` cycles, so simulations of
 * different grids, problems and precisions share every launch, and a
 * simulation joins or leaves at round boundaries.  When a simulation has
 * taken its requested cycles its primitives are copied to the caller's
 * host buffer and its device memory is freed.  A result is bitwise the
 * result of grmhd_step on the same simulation alone. */
typedef struct grmhd_server grmhd_server; /* opaque, library-owned */

typedef struct {
  size_t hbm_budget;           /* bytes of simulation state the server may hold; 0: 90% of
                                  the free device memory at creation */
  long long max_active_zones;  /* admit no request that would take the zones in flight
                                  above this (one is always admitted); 0: no cap */
  int quantum;                 /* cycles per round at most (>= 1) */
  int use_graph;               /* 1: each round replays a CUDA graph of one cycle */
  int policy;                  /* GRMHD_SERVE_FIFO or GRMHD_SERVE_SWF */
} grmhd_server_config;

/* Admission order of waiting requests. */
#define GRMHD_SERVE_FIFO 0 /* arrival order; the oldest waits for room (no overtaking) */
#define GRMHD_SERVE_SWF 1  /* smallest work (zones x cycles) first among those that fit */

typedef struct {
  long long id;                 /* the caller's request id */
  int status;                   /* GRMHD_OK; GRMHD_ERR_INVERSION: the result is there but a
                                  failed zone had no valid neighbour (as grmhd_step reports);
                                  any other code ended the request without a result */
  long long zones, steps;       /* interior zones, cycles taken */
  double t_arrival, t_admit, t_done; /* server clock (seconds): arrival as submitted,
                                  admission (state on the device), result in host memory */
  grmhd_stats stats;            /* the simulation's final statistics */
} grmhd_server_result;

typedef struct {
  double now;                   /* server clock (seconds since creation) */
  long long submitted, completed, failed, rounds; /* completed: with a result */
  double zone_cycles;           /* interior zone-cycles advanced */
  double busy_seconds;          /* wall time with rounds in flight */
  size_t bytes_in_use, peak_bytes, budget;
  int active, pending, peak_active;
  long long launches;           /* kernels launched by the rounds */
} grmhd_server_stats;

/* Start a server on the current device (its thread makes that device
 * current).  cfg == NULL: defaults (budget 90% of free memory, no zone
 * cap, quantum 8, graphs on, FIFO). */
int grmhd_server_create(const grmhd_server_config *cfg, grmhd_server **out);

/* Submit one simulation: grid, metric and parameters as grmhd_create;
 * P_in: host primitives, interior ([8][n3][n2][n1]) or with ghosts
 * (in_ghosts = 1; needed for FIXED boundaries); P_out: host buffer for the
 * result, interior or with ghosts (out_ghosts).  The caller keeps both
 * buffers alive and untouched until the request's result has been polled.
 * t_arrival: the request's arrival on the server clock (a negative value:
 * now); time-to-result is counted from it.  Returns at once; a request
 * whose footprint exceeds the whole budget is refused (GRMHD_ERR_NOMEM),
 * invalid arguments give GRMHD_ERR_INVALID. */
int grmhd_server_submit(grmhd_server *srv, long long id, const grmhd_grid *grid,
                        const grmhd_metric *metric, const grmhd_params *params,
                        const double *P_in, int in_ghosts, double *P_out, int out_ghosts,
                        long long nsteps, double t_arrival);

/* grmhd_server_submit for a simulation that evolves electron entropies
 * (params->electrons.model != 0; grmhd_server_submit refuses those): K_in
 * and K_out are the host entropies (kappa_tot, kappa_e) in and out, with
 * the ghosts as P_in and P_out, kept alive by the caller like them. */
int grmhd_server_submit_electrons(grmhd_server *srv, long long id, const grmhd_grid *grid,
                                  const grmhd_metric *metric, const grmhd_params *params,
                                  const double *P_in, const double *K_in, int in_ghosts,
                                  double *P_out, double *K_out, int out_ghosts, long long nsteps,
                                  double t_arrival);

/* Move up to max finished requests into res (oldest first), waiting up to
 * wait_ms milliseconds for the first; returns how many (>= 0) or an
 * error code. */
int grmhd_server_poll(grmhd_server *srv, grmhd_server_result *res, int max, int wait_ms);

/* Wait until every submitted request has finished (results stay to be
 * polled), at most timeout_ms (< 0: no limit); GRMHD_ERR_CUDA on timeout. */
int grmhd_server_drain(grmhd_server *srv, int timeout_ms);

int grmhd_server_get_stats(grmhd_server *srv, grmhd_server_stats *out);

/* Seconds on the server clock. */
double grmhd_server_now(grmhd_server *srv);

/* Stop the thread (requests not finished are dropped) and free everything.
 * NULL is accepted. */
int grmhd_server_destroy(grmhd_server *srv);

/* ---- Domain decomposition: one grid split into blocks ----
 *
 * The paper scales by splitting the grid into mesh blocks, one per node
 * ("Scaling" section), and tests that the evolution does not depend on the
 * split (end of its "Tests" section).  A decomposed grid here is a set of
 * blocks of one global grid advanced together on the current device: each
 * block fills the ghosts it shares with a neighbour from that neighbour's
 * edge zones, in the order of the global ghost fill; the blocks share one
 * CFL time step (the signal-speed maxima are combined before it is taken);
 * and a failed zone at a block edge averages over the same neighbours as in
 * the whole grid.  The result is bitwise that of grmhd_create/grmhd_step on
 * the undecomposed grid.  The exchange step is the one a multi-GPU split
 * would carry between devices. */
typedef struct grmhd_decomp grmhd_decomp; /* opaque, library-owned */

/* Split the global grid into nblocks[0] x nblocks[1] x nblocks[2] blocks of
 * as equal sizes as possible (each split direction needs >= 3 zones per
 * block); grid, metric and params as grmhd_create.  stream: as grmhd_create
 * (every call of this object is ordered on it). */
int grmhd_decomp_create(const grmhd_grid *grid, const grmhd_metric *metric,
                        const grmhd_params *params, const int nblocks[3], void *stream,
                        grmhd_decomp **out);

int grmhd_decomp_destroy(grmhd_decomp *dc);

/* Host primitives of the global grid, interior ([8][n3][n2][n1]) or with
 * ghosts ([8][n3+6][n2+6][n1+6]; needed for FIXED boundaries); the ghosts
 * are then filled as grmhd_set_prims fills them.  Synchronous. */
int grmhd_decomp_set_prims(grmhd_decomp *dc, const double *P, int with_ghosts);

/* The global primitives into host memory, interior or with ghosts. */
int grmhd_decomp_get_prims(grmhd_decomp *dc, double *P, int with_ghosts);

/* The global electron entropies (kappa_tot, kappa_e), [2][...] as
 * grmhd_set_electrons, host memory; set them after the primitives.
 * GRMHD_ERR_INVALID: the grid evolves no electrons. */
int grmhd_decomp_set_electrons(grmhd_decomp *dc, const double *K, int with_ghosts);
int grmhd_decomp_get_electrons(grmhd_decomp *dc, double *K, int with_ghosts);

/* Advance nsteps cycles, as grmhd_step (stats: the blocks' counters summed). */
int grmhd_decomp_step(grmhd_decomp *dc, int nsteps, grmhd_stats *stats);

/* Synchronise and read the statistics; check != 0 also reports, as
 * grmhd_step does, GRMHD_ERR_INVERSION / GRMHD_ERR_DT since the last check. */
int grmhd_decomp_get_stats(grmhd_decomp *dc, grmhd_stats *stats, int check);

/* Name of an error code (the error convention of this interface; the
 * paper has no counterpart). */
const char *grmhd_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* GRMHD_H */
