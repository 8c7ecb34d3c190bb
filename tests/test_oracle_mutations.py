"""Planted mistakes in the oracle, each of which a pin must catch.

A pin that no plausible mistake can fail proves nothing about the oracle.
Each case copies oracle/grmhd_oracle.cpp, plants one mistake of the kinds a
transcription makes (a dropped term, a wrong sign, a transposed index, a
wrong constant or branch), builds the copy with the oracle's own compiler
flags and runs the pins named beside it against that build (ORACLE_LIB).
The case passes when those pins fail.  CPU only; the oracle's own build is
not touched.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "grmhd_oracle.cpp")

SCHEME = "tests/test_oracle_scheme.py"
PHYSICS = "tests/test_oracle_physics.py"
GEOMETRY = "tests/test_oracle_geometry.py"
RECON = "tests/test_oracle_recon.py"
DRIFT = "tests/test_oracle_floors_drift.py"
ELEC = "tests/test_oracle_electrons.py"
BOUNDARIES = "tests/test_oracle_boundaries.py"
FIXUP_DT = "tests/test_oracle_fixup_dt.py"

# (name, text in the oracle source (exactly once), planted replacement, pins)
MUTATIONS = [
    # local Lax-Friedrichs: the dissipation added instead of subtracted
    ("llf_dissipation_sign", "FL[v] + FR[v] - ctop * (UR[v] - UL[v])",
     "FL[v] + FR[v] + ctop * (UR[v] - UL[v])", [SCHEME]),
    # stress-energy: magnetic pressure dropped from the total pressure
    ("ptot_without_bsq", "real ptot = pgas + 0.5 * s.bsq;", "real ptot = pgas;", [PHYSICS]),
    # energy flux: the rest mass subtracted twice instead of removed
    ("rest_mass_sign", "F[UU] = T[0] + F[RHO];", "F[UU] = T[0] - F[RHO];", [PHYSICS]),
    # fast speed: c_ms^2 = cs^2 + va^2 - cs^2 va^2 with the wrong sign
    ("fast_speed_sign", "real cms2 = cs2 + va2 - cs2 * va2;",
     "real cms2 = cs2 + va2 + cs2 * va2;", [PHYSICS]),
    # MC limiter: the factor 2 of the one-sided slopes dropped
    ("mc_factor", "rabs(2.0 * dm)", "rabs(dm)", [RECON]),
    # WENO5: the linear weights of the high face swapped
    ("weno5_linear_weights", "real a0 = 0.1 / e0, a1 = 0.6 / e1, a2 = 0.3 / e2;",
     "real a0 = 0.3 / e0, a1 = 0.6 / e1, a2 = 0.1 / e2;", [RECON]),
    # flux-CT: one of the four EMF terms with the wrong sign
    ("emf_term_sign", "- F2[B1 * N + c] - F2[B1 * N + im]);",
     "- F2[B1 * N + c] + F2[B1 * N + im]);", [SCHEME]),
    # geometric source: the connection's upper and a lower index transposed
    ("connection_index", "conn[(la * 4 + nu) * 4 + ka]", "conn[(nu * 4 + la) * 4 + ka]",
     [SCHEME + "::test_torus_equilibrium_residual_second_order"]),
    # geometric source with the wrong sign
    ("source_sign", "dU[UU + nu] = acc * g.gdet;", "dU[UU + nu] = -acc * g.gdet;",
     [SCHEME + "::test_torus_equilibrium_residual_second_order"]),
    # 1D_W: v^2(W) with (B^2 + W) for (B^2 + 2W)
    ("inversion_vsq", "q.QdB * q.QdB * (q.Bsq + 2.0 * W)) / (BW * BW * W2)",
     "q.QdB * q.QdB * (q.Bsq + W)) / (BW * BW * W2)", [PHYSICS]),
    # 1D_W: the spatial projection of Q with the wrong sign
    ("inversion_projection", "(g.gcon[i][j] - g.gcon[i][0] * g.gcon[j][0] / g.gcon[0][0])",
     "(g.gcon[i][j] + g.gcon[i][0] * g.gcon[j][0] / g.gcon[0][0])", [PHYSICS]),
    # Kerr-Schild metric: g_tr with the wrong sign
    ("kerr_schild_gtr_sign", "ks[0][1] = 2.0 * r / sig;", "ks[0][1] = -2.0 * r / sig;", [GEOMETRY]),
    # modified Kerr-Schild theta(X2) with h for 1 - h
    ("mks_theta_map", "double th = M_PI * X[2] + 0.5 * (1.0 - h) * std::sin(2.0 * M_PI * X[2]);",
     "double th = M_PI * X[2] + 0.5 * (1.0 + h) * std::sin(2.0 * M_PI * X[2]);", [GEOMETRY]),
    # predictor-corrector: the predictor takes the full step
    ("predictor_full_step", "PHASE(2);\n  int bad = advance_stage(S, S->P, S->P, S->Ph, 0.5 * dt,",
     "PHASE(2);\n  int bad = advance_stage(S, S->P, S->P, S->Ph, dt,",
     [SCHEME + "::test_linear_mode_second_order"]),
    # bounds: the beta bound's u without the factor 2 of P_b = b^2/2
    ("beta_bound_factor", "BETA_MIN * s.bsq / (2.0 * (gam - 1.0))",
     "BETA_MIN * s.bsq / (gam - 1.0)", [PHYSICS]),
    # drift-frame bounds: the field-aligned part added instead of removed
    ("drift_projection_sign", "(Pc[U1 + i] - (udB / Bsq) * Pc[B1 + i])",
     "(Pc[U1 + i] + (udB / Bsq) * Pc[B1 + i])", [DRIFT]),
    # electron entropy flux: the LLF term with the wrong sign
    ("electron_llf_sign", "- ctop * (dR * KR[q] - dL * KL[q])",
     "+ ctop * (dR * KR[q] - dL * KL[q])", [ELEC]),
    # electron heating with the wrong sign
    ("heating_sign", "(ktot_new - ktot_adv);", "(ktot_adv - ktot_new);", [ELEC]),
    # Kawazura: the exponential taken in T_p/T_e instead of T_e/T_p
    ("kawazura_temperature_ratio", "rexp(-0.1 / trat)", "rexp(-0.1 * trat)", [ELEC]),
    # Howes: c3 with the wrong sign of its log term
    ("howes_c3_sign", "18.0 + 5.0 * lt", "18.0 - 5.0 * lt", [ELEC]),
    # Werner: (s/5)/(1 + s/5) for (s/5)/(2 + s/5)
    ("werner_constant", "(s / 5.0) / (2.0 + s / 5.0)", "(s / 5.0) / (1.0 + s / 5.0)", [ELEC]),
    # Rowan: the exponent 3.3 rounded to 3
    ("rowan_exponent", "rpow(1.0 - r, 3.3)", "rpow(1.0 - r, 3.0)", [ELEC]),
    # electron bounds: T_p/T_e's lower and upper limits swapped
    ("electron_bounds_swapped", "real kmax = kk / (a + e.tpte_min * b);",
     "real kmax = kk / (a + e.tpte_max * b);", [ELEC]),
    # entropy bound: u set with (gamma - 1) multiplied instead of divided
    ("entropy_bound_formula", "P[UU] = KTOT_MAX * rpow(P[RHO], e.gam) / (e.gam - 1.0);",
     "P[UU] = KTOT_MAX * rpow(P[RHO], e.gam) * (e.gam - 1.0);", [ELEC]),
    # electron fixup: the neighbours' kappa_tot averaged instead of kappa_e
    ("electron_fixup_index", "if (S->elec) sumk += Kout[N + nb];", "if (S->elec) sumk += Kout[nb];",
     [ELEC]),
    # 4-velocity: u^t = gamma alpha for gamma/alpha
    ("ut_lapse", "ucon[0] = gamma / g.alpha;", "ucon[0] = gamma * g.alpha;", [PHYSICS]),
    # b^i = (B^i + b^t u^i)/u^t with the wrong sign
    ("bcon_sign", "s.bcon[i] = (P[B1 + i - 1] + s.bcon[0] * s.ucon[i]) / s.ucon[0];",
     "s.bcon[i] = (P[B1 + i - 1] - s.bcon[0] * s.ucon[i]) / s.ucon[0];", [PHYSICS]),
    # induction flux b^j u^d - b^d u^j transposed
    ("induction_flux_order", "s.bcon[j] * s.ucon[dir] - s.bcon[dir] * s.ucon[j]",
     "s.bcon[dir] * s.ucon[j] - s.bcon[j] * s.ucon[dir]", [PHYSICS]),
    # signal speeds: the wrong sign of b in one root
    ("vchar_root", "real v1 = (-qb + disc) / (2.0 * qa);", "real v1 = (qb + disc) / (2.0 * qa);",
     [PHYSICS]),
    # 1D_W: the rest-mass term of w - rho with the wrong sign
    ("w_minus_rho_sign", "return Wp * (1.0 - vsq) - q.D * vsq * sq / (1.0 + sq);",
     "return Wp * (1.0 - vsq) + q.D * vsq * sq / (1.0 + sq);", [PHYSICS]),
    # Kerr-Schild g_phiphi without its factor 2
    ("kerr_schild_gphiphi", "ks[3][3] = s2 * (sig + a * a * s2 * (1.0 + 2.0 * r / sig));",
     "ks[3][3] = s2 * (sig + a * a * s2 * (1.0 + r / sig));", [GEOMETRY]),
    # bounds: sigma's limit multiplied instead of divided
    ("sigma_bound", "real rmin_sig = s.bsq / BSQ_OVER_RHO_MAX;",
     "real rmin_sig = s.bsq * BSQ_OVER_RHO_MAX;", [PHYSICS]),
    # drift-frame bounds: the drift Lorentz factor inverted
    ("drift_lorentz_factor", "real f = 1.0 / rsqrt_(1.0 + upar2);", "real f = rsqrt_(1.0 + upar2);",
     [DRIFT]),
    # CFL: the per-direction limits combined by a maximum instead of a sum
    ("cfl_combination", "inv += 1.0 / ndt;", "inv = (1.0 / ndt > inv) ? 1.0 / ndt : inv;",
     [SCHEME + "::test_uniform_dt_closed_form"]),
    # fixup: failed neighbours included in the mean
    ("fixup_uses_failed_zones",
     "if (S->pflag[nb] != INV_OK) continue;\n              for (int v = 0; v < 5; v++)",
     "for (int v = 0; v < 5; v++)", [SCHEME + "::test_torus_equatorial_symmetry"]),
    # fixup: only the six face neighbours averaged
    ("fixup_six_face_neighbours", "if (di == 0 && dj == 0 && dk == 0) continue;",
     "if (di * di + dj * dj + dk * dk != 1) continue;", [FIXUP_DT]),
    # fixup: the failed zone's own values counted in the mean
    ("fixup_mean_includes_centre", "if (di == 0 && dj == 0 && dk == 0) continue;",
     "if (di == 0 && dj == 0 && dk == 0) {\n                for (int v = 0; v < 5; v++) "
     "sum[v] += Pout[v * N + c];\n                cnt++;\n                continue;\n"
     "              }", [FIXUP_DT]),
    # time step: the growth limit 2 instead of 1.3
    ("dt_growth_limit", "dt > 1.3 * S->dt_prev) dt = 1.3 * S->dt_prev;",
     "dt > 2.0 * S->dt_prev) dt = 2.0 * S->dt_prev;", [FIXUP_DT]),
    # polar ghosts: B^2 not turned over
    ("polar_b2_not_flipped",
     "copy_zone(S, P, K, d, IDX(S, i, NG + g, k));\n          P[U2 * N + d] = -P[U2 * N + d];\n"
     "          P[B2 * N + d] = -P[B2 * N + d];",
     "copy_zone(S, P, K, d, IDX(S, i, NG + g, k));\n          P[U2 * N + d] = -P[U2 * N + d];",
     [BOUNDARIES]),
    # polar ghosts mirrored one zone off
    ("polar_mirror_offset", "copy_zone(S, P, K, d, IDX(S, i, NG + g, k));",
     "copy_zone(S, P, K, d, IDX(S, i, NG + g + 1, k));", [BOUNDARIES]),
    # outflow ghosts: the inflow check with the wrong sign
    ("outflow_ghost_inflow_sign", "if (P[U1 * N + d] > 0.0) P[U1 * N + d] = 0.0;",
     "if (P[U1 * N + d] < 0.0) P[U1 * N + d] = 0.0;", [BOUNDARIES]),
    # outflow faces: outflow zeroed instead of inflow
    ("outflow_face_inflow_sign", "if (S->F[0][RHO * N + id] > 0.0) {",
     "if (S->F[0][RHO * N + id] < 0.0) {", [BOUNDARIES]),
    # predictor-corrector: the corrector's geometric source at P^n, not P^(n+1/2)
    ("corrector_source_state", "bad += advance_stage(S, S->P, S->Ph, S->P, dt,",
     "bad += advance_stage(S, S->P, S->P, S->P, dt,",
     [SCHEME + "::test_time_integration_second_order_in_curved_space"]),
    # periodic X3 ghosts filled from the first zone instead of the last
    ("x3_periodic_not_wrapped",
     "copy_zone(S, P, K, IDX(S, i, j, kg), IDX(S, i, j, wrap_index(kg, n3)));\n"
     "        else if (S->bc[2][0] == BC_OUTFLOW)",
     "copy_zone(S, P, K, IDX(S, i, j, kg), IDX(S, i, j, NG));\n"
     "        else if (S->bc[2][0] == BC_OUTFLOW)",
     [SCHEME + "::test_conservation_periodic_flat_3d"]),
    # WENO5: a smoothness indicator's second term with 1/2 for 1/4
    ("weno5_indicator_coefficient", "  real e0 = eps + ((13.0 / 12.0) * t * t + 0.25 * s * s);",
     "  real e0 = eps + ((13.0 / 12.0) * t * t + 0.5 * s * s);", [RECON]),
    # LLF: the left state's face value taken from the wrong side of its zone
    ("face_states_swapped", "PL[v] = S->Rz[v * N + c - st];", "PL[v] = S->Lz[v * N + c - st];",
     [SCHEME + "::test_linear_mode_second_order"]),
    # LLF: the left-going speeds' sign in c_max
    ("llf_cmin_sign", "real cmin = rmax(rmax(real(0.0), -vminL), -vminR);",
     "real cmin = rmax(rmax(real(0.0), vminL), vminR);",
     [SCHEME + "::test_torus_equilibrium_residual_second_order"]),
    # CFL: the Courant factor dropped
    ("cfl_factor_missing", "double ndt = S->cfl * S->dx[d] / ct;", "double ndt = S->dx[d] / ct;",
     [SCHEME + "::test_uniform_dt_closed_form"]),
    # flux-CT: emf1 averaged over the wrong neighbour
    ("emf1_neighbour",
     "e1[c] = 0.25 * (F2[B3 * N + c] + F2[B3 * N + km] - F3[B2 * N + c] - F3[B2 * N + jm]);",
     "e1[c] = 0.25 * (F2[B3 * N + c] + F2[B3 * N + jm] - F3[B2 * N + c] - F3[B2 * N + jm]);",
     [SCHEME]),
    # electron fluxes: the two sides' densities swapped in the LLF term
    ("electron_densities_swapped", "real dL = PL[RHO] * sL.ucon[0], dR = PR[RHO] * sR.ucon[0];",
     "real dR = PL[RHO] * sL.ucon[0], dL = PR[RHO] * sR.ucon[0];", [ELEC]),
    # heating fits: T_p/T_e clamped inside the range the bounds allow
    ("temperature_ratio_clamp", "trat = rmin(rmax(trat, real(1.0e-20)), real(1.0e20));",
     "trat = rmin(rmax(trat, real(1.0e-2)), real(1.0e2));", [ELEC]),
    # electron entropies carried from the source stage's kappa, not kappa^n
    ("electron_advection_state", "real Uk = Ui[RHO] * Ki[o + c] + dtp * (0.0 - divk);",
     "real Uk = Ui[RHO] * Ks[o + c] + dtp * (0.0 - divk);",
     [ELEC + "::test_passive_electron_entropy_is_conserved_in_compressive_flow"]),
    # outer boundary: the mass inflow zeroed but the entropies' flux kept
    ("outflow_electron_flux_kept",
     "          if (S->F[0][RHO * N + id] < 0.0) {\n            S->F[0][RHO * N + id] = 0.0;\n"
     "            if (S->elec)\n              for (int q = 0; q < 2; q++) S->FK[0][q * N + id] = 0.0;",
     "          if (S->F[0][RHO * N + id] < 0.0) {\n            S->F[0][RHO * N + id] = 0.0;",
     [ELEC + "::test_uniform_electron_entropy_stays_uniform_on_the_torus"]),
    # bounds: the density floor reported as the internal-energy floor
    ("floor_flag_swapped",
     "if (P[RHO] < rho_fl) { P[RHO] = rho_fl; flags |= FF_RHO_GEOM; }",
     "if (P[RHO] < rho_fl) { P[RHO] = rho_fl; flags |= FF_U_GEOM; }", [PHYSICS]),
    # ghost fill: the electron entropies not copied into the ghosts
    ("electron_ghosts_not_filled",
     "    for (int q = 0; q < 2; q++) K[q * S->ntot + dst] = K[q * S->ntot + src];", "    (void)K;",
     [ELEC]),
    # electrons: kappa_tot reset from u/rho instead of u/rho^gamma
    ("ktot_reset_formula", "  K[0] = (e.gam - 1.0) * P[UU] / rpow(P[RHO], e.gam);",
     "  K[0] = (e.gam - 1.0) * P[UU] / P[RHO];", [ELEC]),
    # 1D_W: a negative u reported as success
    ("negative_u_accepted", "  if (uu < 0.0) return INV_U_NEG;", "  if (uu < 0.0) return INV_OK;",
     [ELEC]),
    # b^2 without its time component
    ("bsq_without_time_part", "for (int m = 0; m < 4; m++) s.bsq += s.bcon[m] * s.bcov[m];",
     "for (int m = 1; m < 4; m++) s.bsq += s.bcon[m] * s.bcov[m];", [PHYSICS]),
    # outflow ghosts: B copied without the sqrt(-g) rescaling
    ("outflow_b_not_rescaled",
     "for (int b = B1; b <= B3; b++) P[b * N + d] *= rescale;\n          if (P[U1 * N + d] > 0.0)",
     "(void)rescale;\n          if (P[U1 * N + d] > 0.0)", [BOUNDARIES]),
]


def _source():
    with open(SRC) as f:
        return f.read()


def test_every_mutation_applies_once():
    src = _source()
    names = [m[0] for m in MUTATIONS]
    assert len(set(names)) == len(names)
    for name, old, _new, _pins in MUTATIONS:
        assert src.count(old) == 1, name


def _run_mutation(workdir, name, old, new, pins):
    """Build the oracle with one planted mistake and run its pins against
    it; returns the pins' pytest exit code and output."""
    src = _source()
    assert src.count(old) == 1, name
    cpp = os.path.join(workdir, name + ".cpp")
    so = os.path.join(workdir, "lib" + name + ".so")
    with open(cpp, "w") as f:
        f.write(src.replace(old, new))
    subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                    "-o", so, cpp], check=True)
    env = dict(os.environ, ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        "-m", "not gpu", *pins], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    return r.returncode, r.stdout[-2000:] + r.stderr[-2000:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """Every case built and run at once (independent processes)."""
    workdir = str(tmp_path_factory.mktemp("mutations"))
    workers = max(1, min(8, os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        futures = {m[0]: ex.submit(_run_mutation, workdir, *m) for m in MUTATIONS}
        return {name: f.result() for name, f in futures.items()}


@pytest.mark.parametrize("name", [m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(outcomes, name):
    rc, out = outcomes[name]
    # exit code 1: tests ran and failed (2-5 would be an error of the run itself)
    assert rc == 1, "no pin caught %s:\n%s" % (name, out)
    assert " failed" in out
