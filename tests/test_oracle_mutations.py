"""Plant plausible mistakes in copies of the oracle and check that a pin
catches each one (a flipped sign, a dropped Jacobian term, a transposed
operand, a wrong tilt or Lorentz sign, a broken selection order, a
mis-scaled scattering or energy-loss term)."""
import os
import subprocess

import pytest

from oracle import oracle as O
import test_oracle_pins as P
import test_oracle_refit_pins as R
import test_oracle_residual_pins as Q
import test_oracle_alignment_pins as M

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "trd_oracle.c")

PINNED = [
    ("curvature sign", "const double rho = drho_dk * k;", "const double rho = -drho_dk * k;"),
    ("dropped dy/dk term", "J[0][4] = dx * dh_df1 * drho_dk * dx;", "J[0][4] = 0.0;"),
    ("transposed operand in J C J^T", "s += t[i][k] * J[j][k];", "s += t[i][k] * J[k][j];"),
    ("chord slope", "const double h = (f0 + f1) / rs;", "const double h = (f0 + f1) / (2.0 * rs);"),
    ("arc series", "return 1.0 + w2 / 6.0 + 3.0 * w2 * w2 / 40.0;", "return 1.0 + w2 / 3.0 + 3.0 * w2 * w2 / 40.0;"),
    ("rotation dsnp/dy sign", "J[2][0] = -rho * sd;", "J[2][0] = rho * sd;"),
    ("rotation dy/dy inverted", "J[0][0] = r / rn;", "J[0][0] = rn / r;"),
    ("pad tilt sign", "static double tilt_tan(int l) { return tan((l % 2 == 0 ? 1.0 : -1.0)",
     "static double tilt_tan(int l) { return tan((l % 2 == 0 ? -1.0 : 1.0)"),
    ("tilt term in residual", "o->r[0] = ytl - (st[2] - tt * (st[3] - ztl));",
     "o->r[0] = ytl - (st[2] + tt * (st[3] - ztl));"),
    ("dropped tilt in S01", "o->S[1] = c[1] - tt * c[2] + vyz;", "o->S[1] = c[1] + vyz;"),
    ("chi2 cross-term sign", "o->chi2 = (o->S[2] * o->r[0] * o->r[0] - 2.0 * o->S[1]",
     "o->chi2 = (o->S[2] * o->r[0] * o->r[0] + 2.0 * o->S[1]"),
    ("gain index", "K[i][a] = CHt[i][0] * Si[0][a] + CHt[i][1] * Si[1][a];",
     "K[i][a] = CHt[i][0] * Si[a][0] + CHt[i][1] * Si[a][0];"),
    ("deflection prediction", "const double dy_pred = kDriftLength * u;", "const double dy_pred = kDriftLength * f;"),
    ("Lorentz angle sign", "static double lorentz_tan(double bz) { return tan((bz >= 0 ? 1.0 : -1.0)",
     "static double lorentz_tan(double bz) { return tan((bz >= 0 ? -1.0 : 1.0)"),
    ("selection keeps the worst", "if (a->score < b->score) return -1;\n    if (a->score > b->score) return 1;",
     "if (a->score > b->score) return -1;\n    if (a->score < b->score) return 1;"),
    ("missing budget off by one", "if (work[hi].nmiss < P->max_missing)", "if (work[hi].nmiss <= P->max_missing)"),
    ("association ignores the ids", "return seed_trig < 0 || !T->trig || T->trig[j] < 0 || T->trig[j] == seed_trig;",
     "return 1;"),
    ("road uses n^2", "const double s[4] = {P->n_sigma_road - ny,", "const double s[4] = {P->n_sigma_road * P->n_sigma_road - ny,"),
    # the TRD-only refit (Sec. 2, step 3)
    ("refit prior not widened", "for (int i = 0; i < 5; ++i) h.c[ci(i, i)] = cov_scale * in_cdiag[i];",
     "for (int i = 0; i < 5; ++i) h.c[ci(i, i)] = in_cdiag[i];"),
    ("refit loss taken with the outward sign", "if (P->material_on && material_dir(h.st, h.c, -1.0)) { fail = 1; break; }",
     "if (P->material_on && material_dir(h.st, h.c, 1.0)) { fail = 1; break; }"),
    ("refit skips the outermost update", "for (int l = ltop; l >= 0 && !fail; --l) {",
     "for (int l = ltop - 1; l >= 0 && !fail; --l) {"),
    ("refit update with the next layer's tilt", "h.chi2 += ora_update(h.st, h.c, l, m5, 0);",
     "h.chi2 += ora_update(h.st, h.c, l + 1, m5, 0);"),
    ("refit stays in its sector", "            target = T->ch[j] / (ORA_NSTACK * ORA_NLAYER);",
     "            target = h.sector;"),
    # residuals in TPC sub-volumes and the distortion vector (Sec. 2, steps 4-5)
    ("residual sign", "out[0] = (double)ycl - my;", "out[0] = my - (double)ycl;"),
    ("y slope without 1/cos", "out[2] = f / r;", "out[2] = f;"),
    ("z slope without 1/cos", "out[3] = tl / r;", "out[3] = tl;"),
    ("combination drops the TRD refit", "const double b0 = g[0][0] + g[1][0], b1 = g[0][1] + g[1][1];",
     "const double b0 = g[0][0] + g[0][0], b1 = g[0][1] + g[0][1];"),
    ("combined variance of one refit", "out[4] = W11 / dW;", "out[4] = c[0][0];"),
    ("voxel side from y", "const int side = z < 0.0f ? 1 : 0;", "const int side = y < 0.0f ? 1 : 0;"),
    ("y bin without offset", "const float v = u + T;", "const float v = u;"),
    ("solve sign of Dx", "const double dx = -(n * (S[7] + S[8])", "const double dx = (n * (S[7] + S[8])"),
    ("solve drops the angular mean", "o[1] = (S[5] + S[1] * dx) / n;", "o[1] = S[5] / n;"),
    # the material step (Sec. 3, "energy loss"; constants are a reading)
    ("scattering on snp without cos^2", "c[ci(2, 2)] += th2 * r * r * t2;", "c[ci(2, 2)] += th2 * r * t2;"),
    ("scattering tgl-q2pt sign", "c[ci(4, 3)] += th2 * t * t2 * k;", "c[ci(4, 3)] -= th2 * t * t2 * k;"),
    ("scattering q2pt without tgl^2", "c[ci(4, 4)] += th2 * t * t * k * k;", "c[ci(4, 4)] += th2 * k * k;"),
    ("path without 1/cos(phi)", "const double path = sqrt(t2) / r;", "const double path = sqrt(t2);"),
    ("energy loss halved", "const double de = ora_bethe(bg) * xrho * 1e-3;",
     "const double de = 0.5 * ora_bethe(bg) * xrho * 1e-3;"),
    ("loss Jacobian without the Bethe slope", "(ora_bethe_dbg(bg) * dp[a] / kMassPion * path",
     "(0.0 * dp[a] / kMassPion * path"),
    ("loss Jacobian without the path term", "+ ora_bethe(bg) * dpath[a]);", ");"),
    ("Bethe slope sign", "const double d_inv_b2 = -2.0 / (bg2 * bg);", "const double d_inv_b2 = 2.0 / (bg2 * bg);"),
    # misalignment and the field map (Sec. 3)
    ("no linear extrapolation to the tracklet radius", "        sx[2] += dx * f / r;", "        sx[2] += 0.0 * dx * f / r;"),
    ("no precise transport before the update", "if (T->x) (void)fprop(h.st, h.c, (double)T->x[x->id], P, NULL);", ""),
    ("chamber radius ignored", "if (P->chamber_x && (double)P->chamber_x[*chamber] != xl) {", "if (0) {"),
    ("step field at the start point", "    return field_at(P, hypot(st[1] + h, st[2] + h * f / r), st[3] + h * st[5] / r);",
     "    return field_at(P, hypot(st[1], st[2]), st[3]);"),
    ("field map axes swapped", "    return (1 - wz) * ((1 - wr) * F[j * nr + i] + wr * F[j * nr + i + 1]) +",
     "    return (1 - wr) * ((1 - wz) * F[j * nr + i] + wz * F[j * nr + i + 1]) +"),
    ("refit at the nominal radius", "const double xl = (j >= 0 && T->x) ? (double)T->x[j] : layer_x(l);",
     "const double xl = layer_x(l);"),
]

PINS = [
    lambda: P.test_bethe_slope_matches_finite_differences(),
    lambda: P.test_material_scattering_matches_monte_carlo_of_two_angles(False),
    lambda: P.test_material_energy_change_is_the_bethe_loss_over_the_path(False),
    lambda: P.test_material_covariance_transport_is_the_jacobian_of_the_state_map(False),
    lambda: P.test_helix_matches_circle_intersection(12.6),
    lambda: P.test_helix_matches_circle_intersection(-25.0),
    lambda: P.test_transport_jacobian_matches_finite_differences(0.5),
    lambda: P.test_transport_jacobian_small_curvature_series_branch(),
    lambda: P.test_transport_covariance_is_j_c_jt_and_stays_pd(),
    lambda: P.test_rotation_jacobian_matches_finite_differences(0.5),
    lambda: P.test_rotation_round_trip_is_identity(),
    lambda: P.test_kalman_update_equals_information_form(0),
    lambda: P.test_pad_tilt_sign_residual_vanishes_on_tilted_measurement(),
    lambda: P.test_zero_noise_truth_is_recovered_exactly(),
    lambda: P.test_zero_noise_with_pad_rows_assigns_truth(),
    lambda: P.test_dy_gate_at_four_sigma(),
    lambda: P.test_road_boundary_at_n_sigma(),
    lambda: P.test_association_never_crosses_interactions(),
    lambda: P.test_tiny_efficiency_and_purity(),
    lambda: P.test_greedy_n1_takes_best_chi2_each_layer(),
    lambda: P.test_beam_search_equals_exhaustive_enumeration(),
    lambda: R.test_refit_equals_map_least_squares_without_material(100.0, 0.5, 0.05),
    lambda: R.test_refit_recovers_noiseless_truth(),
    lambda: R.test_refit_pulls_are_unit_normal(),
    lambda: R.test_inward_refit_undoes_the_outward_material(),
    lambda: R.test_refit_output_frame_is_the_layer0_sector(),
    lambda: R.test_refit_skips_unmatched_and_invalid_tracks(),
    lambda: Q.test_voxel_of_hand_placed_clusters(),
    lambda: Q.test_no_distortion_exact_refits_give_zero_residuals(),
    lambda: Q.test_residuals_follow_the_injected_field(),
    lambda: Q.test_combined_estimate_has_unit_pulls(),
    lambda: Q.test_voxel_solve_equals_least_squares(),
    lambda: Q.test_map_recovers_a_uniform_displacement(),
    lambda: M.test_misaligned_truth_is_found_with_the_radii_and_not_without(),
    lambda: M.test_state_after_the_last_update_is_the_truth_at_that_radius(),
    lambda: M.test_a_layer_without_tracklet_ends_at_the_chamber_radius(),
    lambda: M.test_nominal_radii_reproduce_the_aligned_follower(),
    lambda: M.test_uniform_field_map_is_the_homogeneous_field(),
    lambda: M.test_field_map_step_agrees_with_runge_kutta(),
    lambda: M.test_refit_at_the_tracklet_radii_recovers_the_truth(),
]


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation '{name}' does not apply"
    mut = tmp_path / (name.replace(" ", "_").replace("/", "_") + ".c")
    mut.write_text(src.replace(old, new))
    so = str(mut) + ".so"
    subprocess.run(["gcc", "-O1", "-fopenmp", "-fPIC", "-shared", "-std=c11", str(mut), "-o", so, "-lm"],
                   check=True)
    return so


def _caught(so):
    with O.use_library(so):
        for pin in PINS:
            try:
                pin()
            except (AssertionError, ValueError, FloatingPointError):
                return True
    return False


@pytest.mark.parametrize("name,old,new", PINNED, ids=[m[0] for m in PINNED])
def test_pins_catch_planted_mistake(tmp_path, name, old, new):
    assert _caught(_build_mutant(tmp_path, name, old, new)), f"no pin caught: {name}"
