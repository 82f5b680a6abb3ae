"""The oracle's pins are strong enough to reject plausible mistakes (CPU):
each case copies the oracle's source, plants one error of the kind a
transcription makes (a dropped term, a wrong sign, a swapped or mistyped
coefficient, a wrong factor), compiles that copy with gcc, and runs the pins
that should catch it against it (in a child process, through the oracle's
UCNS_ORACLE_LIB override); they must fail.  The unmodified oracle passes the
same pins in the ordinary suite.  The oracle's Python parts (the network's
reference oracle/mlp.py, the parameter array and the labels in
oracle/__init__.py) are mutated the same way in a copy of the source tree,
where the pins import the mutated copy.

Left out as equivalent: a ReLU mask taken as >= 0 instead of > 0 (it
differs only at exact zeros), and one Gauss point fewer in the smoothness
indicator of a cubic (on affine cells three points per direction are
already exact, and on trilinear cells neither rule is, so no closed form
tells the two apart)."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ucns_oracle.c")

MUTANTS = [
    ("scheme_mask_sense_inverted", ("(c->mask && !c->mask[i])", "(c->mask && c->mask[i])"),
     "test_scheme_mask_routes_each_cell"),
    ("scheme_mask_of_a_stencil_member", ("(c->mask && !c->mask[i])", "(c->mask && !c->mask[c->sc[i * c->Mc]])"),
     "test_scheme_mask_routes_each_cell"),
    # name, (original text, planted mistake), pins that must catch it
    ("hllc_pressure_dropped", ("F[1 + d] = r * u[d] * un + p * n[d];", "F[1 + d] = r * u[d] * un;"),
     "test_hllc_consistency_contact_upwind_symmetry"),
    ("stokes_factor", ("(a == j ? 2.0 / 3.0 * mu * div : 0.0)", "(a == j ? 1.0 / 3.0 * mu * div : 0.0)"),
     "test_viscous_flux_linear_velocity_uniform_temperature"),
    ("lsq_volume_weight_dropped", ("P[k * M + r] = s * Vm[r];", "P[k * M + r] = s;"),
     "test_k_exact_reconstruction"),
    ("rk3_stage_weights_swapped", ("U1[k] = 0.75 * U0[k] + 0.25 * (U1[k] + dt * R[k]);",
                                   "U1[k] = 0.25 * U0[k] + 0.75 * (U1[k] + dt * R[k]);"),
     "test_ssprk3_stability_polynomial"),
    ("ssp54_digits_transposed", ("{0, 0.368410593050371, 0, 0, 0},", "{0, 0.368410593050317, 0, 0, 0},"),
     "test_ssp54_coefficients_meet_the_order_conditions"),
    ("face_normal_flipped", ("dS[q][d] = gw[ia] * gw[ib] * nrm[d];", "dS[q][d] = -gw[ia] * gw[ib] * nrm[d];"),
     "test_face_area_vectors_point_from_owner_to_neighbour"),
    ("si_second_derivative_weight", ("q.w2 = pow(c->vol[i], 4.0 / 3.0 - 1.0);", "q.w2 = pow(c->vol[i], 2.0 / 3.0 - 1.0);"),
     "test_smoothness_indicator_closed_forms"),
    ("cubic_gradient_entry", ("g[14][0] = y * y;", "g[14][0] = 2 * y * y;"), "test_k_exact_p3"),
    ("wall_mirror_half", ("UR[1 + d] = UL[1 + d] - 2.0 * mn * nh[d];", "UR[1 + d] = UL[1 + d] - mn * nh[d];"),
     "test_walls_free_stream_and_conservation"),
    ("cwenoz_tau_summed", ("    tau /= (double)nv;\n", "\n"), "test_cwenoz_weights_worked_example"),
    ("cwenoz_eps_dropped", ("lam[s] * (1.0 + tau / (c->eps + SI[s]))", "lam[s] * (1.0 + tau / (SI[s] + 1e-300))"),
     "test_cwenoz_weights_worked_example"),
    ("cwenoz_central_candidate_undivided", ("      as[0][k] = t / lam[0];", "      as[0][k] = t;"),
     "test_k_exact_reconstruction"),
    ("hllc_star_speed_pressure_sign", ("double Ss = (pR - pL + rL", "double Ss = (pL - pR + rL"),
     "test_hllc_sod_interface_flux"),
    ("heat_conductivity_inverted", ("kap = mu * cp / Pr;", "kap = mu * cp * Pr;"),
     "test_viscous_flux_heat_conduction_and_rest"),
    ("jump_penalty_dropped", ("+ c->alpha / Lint * (UR[v] - UL[v]) * nh[j];", ";"),
     "test_jump_penalty_on_the_odd_even_mode"),
    ("face_gradient_not_averaged", ("gf[v * 3 + j] = 0.5 * (gL[v][j] + gR[v][j])", "gf[v * 3 + j] = (gL[v][j] + gR[v][j])"),
     "test_viscous_residual_of_a_shear_wave"),
    ("penalty_length_without_periodic_shift", ("double dd = c->cen[3 * nb + d] + shv[d] - c->cen[3 * o + d];",
                                               "double dd = c->cen[3 * nb + d] - c->cen[3 * o + d];"),
     "test_jump_penalty_on_the_odd_even_mode"),
    ("viscous_face_state_one_sided", ("Uf[v] = 0.5 * (UL[v] + UR[v]);", "Uf[v] = UL[v];"),
     "test_jump_penalty_on_the_odd_even_mode"),
    ("viscous_time_step_gamma_dropped", ("c->Pr / (2.0 * c->gam * (1.0 / c->Re));", "c->Pr / (2.0 * (1.0 / c->Re));"),
     "test_cfl_time_step_closed_form"),
    ("dilatational_factor_dropped", ("out[2] = 4.0 / 3.0 * mu * ed / vt;", "out[2] = mu * ed / vt;"),
     "test_dissipation_diagnostics_of_plane_waves"),
    ("tgv_pressure_amplitude", ("(cos(2 * x[0]) + cos(2 * x[1])) / 16.0;", "(cos(2 * x[0]) + cos(2 * x[1])) / 8.0;"),
     "test_tgv_initial_pressure_solves_the_poisson_equation"),
    ("tgv_density_gamma_dropped", ("    r = g * M * M * pr;\n", "    r = M * M * pr;\n"),
     "test_tgv_initial_pressure_solves_the_poisson_equation"),
    ("feature_density_jump_unnormalised", ("F[m] = (U[j] - r) / r;", "F[m] = (U[j] - r);"),
     "test_features_of_linear_density_and_pressure"),
    ("feature_smoothness_scale", ("q = 0.1 * sc[v];", "q = 0.01 * sc[v];"),
     "test_features_of_linear_density_and_pressure"),
    ("feature_energy_scale", ("double sc[5] = {r, r * a, r * a, r * a, r * a * a};",
                              "double sc[5] = {r, r * a, r * a, r * a, r * a};"),
     "test_features_of_linear_density_and_pressure"),
    ("feature_dilatation_unscaled", ("F[30] = c->hh[i] * fabs(dv) / a;", "F[30] = fabs(dv) / a;"),
     "test_features_closed_forms"),
    ("tet_jacobian_power", ("*detJ = a * a * b * det3(v1, v2, v3);", "*detJ = a * b * det3(v1, v2, v3);"),
     "test_geometry_closed_surfaces_and_volume"),
    ("tet_map_last_term", ("+ a * b * cc * e3[d];", "+ a * cc * e3[d];"), "test_face_quadrature_integrates_bilinear_exactly"),
    ("triangle_collapsed_weight", ("dS[q][d] = gw[ia] * gw[ib] * a * n[d];", "dS[q][d] = gw[ia] * gw[ib] * n[d];"),
     "test_face_quadrature_integrates_bilinear_exactly"),
    ("triangle_centroid_rule_area", ("dS[0][d] = 0.5 * n[d];", "dS[0][d] = n[d];"),
     "test_face_quadrature_integrates_bilinear_exactly"),
    ("triangle_collapsed_point", ("x[q][d] = Q[0][d] + a * e1[d] + a * b * e2[d];", "x[q][d] = Q[0][d] + a * e1[d] + b * e2[d];"),
     "test_face_quadrature_integrates_bilinear_exactly"),
    ("central_stencil_shared_nodes_ascending", ("return q->shared - p->shared;", "return p->shared - q->shared;"),
     "test_stencil_membership_hex_lattice"),
    ("directional_search_enters_the_cell", ("if (m < 0 || m == avoid) continue;", "if (m < 0) continue;"),
     "test_stencil_membership_hex_lattice"),
    ("directional_linear_weight", ("lam[s] = dv[s - 1] ? 1.0 / lsum : 0.0;", "lam[s] = dv[s - 1] ? 2.0 / lsum : 0.0;"),
     "test_cwenoz_weights_worked_example"),
    ("nonlinear_weights_not_normalised", ("for (int s = 0; s < st; s++) wt[s] /= wsum;", "for (int s = 0; s < st; s++) wt[s] /= 1.0;"),
     "test_cwenoz_weights_normalised_and_tend_to_linear"),
    ("roe_sound_speed", ("double at = sqrt((g - 1.0) * (Ht - 0.5 * q2));", "double at = sqrt((g - 1.0) * (Ht - q2));"),
     "test_hllc_resolves_an_isolated_shock_exactly"),
    ("roe_weights_swapped", ("ut[d] = (sL * uL[d] + sR * uR[d]) / (sL + sR);", "ut[d] = (sR * uL[d] + sL * uR[d]) / (sL + sR);"),
     "test_hllc_resolves_an_isolated_shock_exactly"),
    ("right_star_energy_sign", ("(Ss - unR) * (Ss + pR / (rR * (SR - unR))));", "(Ss - unR) * (Ss - pR / (rR * (SR - unR))));"),
     "test_hllc_consistency_contact_upwind_symmetry"),
    ("cubic_hessian_entry", ("H[18][3] = z; H[18][4] = y; H[18][5] = x;", "H[18][3] = z; H[18][4] = z; H[18][5] = x;"),
     "test_smoothness_indicator_cubic_on_a_stretched_cell"),
    ("derivative_falling_factorial", ("v *= (double)(e[d] - j);", "v *= (double)(e[d]);"),
     "test_smoothness_indicator_cubic_closed_forms"),
    ("sampled_residual_volume", ("R[v * ns + k] = -s[v] / c->vol[i];", "R[v * ns + k] = -s[v] / c->vol[i] / c->vol[i];"),
     "test_residual_of_sampled_cells_equals_the_full_residual"),
    ("boundary_sides_swapped", ("return c->bc[2 * ax + (s[ax] > 0 ? 1 : 0)];", "return c->bc[2 * ax + (s[ax] > 0 ? 0 : 1)];"),
     "test_supersonic_inflow_outflow"),
    ("integrator_selection_swapped", ("int rc = c->rk == 1 ? orc_ssp54_generic", "int rc = c->rk == 0 ? orc_ssp54_generic"),
     "test_rk_step_composes_the_residual"),
    ("fourth_derivative_index_repeated", ("{0, 1, 3}, {2, 2, 0}, {2, 0, 2}, {0, 2, 2}, {2, 1, 1}, {1, 2, 1}, {1, 1, 2}};",
                                          "{0, 1, 3}, {2, 2, 0}, {2, 0, 2}, {0, 2, 2}, {2, 1, 1}, {1, 2, 1}, {1, 2, 1}};"),
     "test_smoothness_indicator_quartic_closed_form"),
    ("quartic_basis_entry", ("{0, 1, 3},\n    {2, 2, 0}", "{0, 1, 3},\n    {2, 1, 0}"), "test_k_exact_p4"),
    ("p4_directional_candidates_linear", ("c->Kd = c->order == 4 ? 9 : 3;", "c->Kd = 3;"),
     "test_counts_p4_match_benchmark_matrix"),
    ("inflow_state_offset", ("c->uinf[v] = params[17 + v];", "c->uinf[v] = params[16 + v];"),
     "test_supersonic_inflow_outflow"),
    ("time_step_face_missing", ("for (int j = 0; j < c->nfc; j++) asum += face_area", "for (int j = 0; j < c->nfc - 1; j++) asum += face_area"),
     "test_cfl_time_step_closed_form"),
    ("kinetic_energy_half_dropped", ("ke += V * 0.5 * r * (", "ke += V * r * ("),
     "test_dissipation_diagnostics_of_plane_waves"),
    ("velocity_gradient_without_density_term",
     ("gu[a][j] = (gU[(1 + a) * 3 + j] - u[a] * gU[j]) / r;\n  for (int j = 0; j < 3; j++) {\n    double de",
      "gu[a][j] = (gU[(1 + a) * 3 + j]) / r;\n  for (int j = 0; j < 3; j++) {\n    double de"),
     "test_viscous_flux_of_a_general_state"),
    ("face_gradient_owner_only", ("gf[v * 3 + j] = 0.5 * (gL[v][j] + gR[v][j])", "gf[v * 3 + j] = gL[v][j]"),
     "test_residual_independent_of_cell_numbering"),
    ("gauss_weight_doubled", ("w[i] = 1.0 / ((1.0 - z * z) * dp * dp);", "w[i] = 2.0 / ((1.0 - z * z) * dp * dp);"),
     "test_geometry_closed_surfaces_and_volume"),
    ("hex_face_inward", ("{{0,4,7,3},{1,2,6,5}", "{{0,3,7,4},{1,2,6,5}"), "test_geometry_closed_surfaces_and_volume"),
    ("tet_face_inward", ("{{0,2,1},{0,1,3}", "{{0,1,2},{0,1,3}"), "test_geometry_closed_surfaces_and_volume"),
    ("neighbour_orientation_sign", ("c->cs[q->n * c->nfc + q->nlf] = -1;", "c->cs[q->n * c->nfc + q->nlf] = 1;"),
     "test_discrete_conservation"),
    ("hex_map_corners_swapped", ("{{0,0,0},{1,0,0},{1,1,0},{0,1,0}", "{{0,0,0},{1,0,0},{0,1,0},{1,1,0}"),
     "test_geometry_closed_surfaces_and_volume"),
    ("tet_map_edge", ("e2[d] = P[2][d] - P[1][d];\n      e3[d]", "e2[d] = P[2][d] - P[0][d];\n      e3[d]"),
     "test_face_area_vectors_point_from_owner_to_neighbour"),
    ("prism_base_inward", ("{{0,2,1,-1},{3,4,5,-1},{0,1,4,3}", "{{0,1,2,-1},{3,4,5,-1},{0,1,4,3}"),
     "test_geometry_closed_surfaces_and_volume"),
    ("prism_side_face_nodes", ("{1,2,5,4},{2,0,3,5}}", "{1,2,5,4},{2,0,5,3}}"), "test_counts_prisms"),
    ("prism_map_base_derivative", ("db[d] = (1.0 - w) * a * e2 + w * a * f2;", "db[d] = (1.0 - w) * a * e2 + w * f2;"),
     "test_face_quadrature_integrates_bilinear_exactly"),
    ("prism_map_top_triangle", ("T = P[3][d] + a * f1 + a * b * f2;", "T = P[3][d] + a * f1 + b * f2;"),
     "test_face_quadrature_integrates_bilinear_exactly"),
    ("prism_one_triangle", ("(lf < 2 ? 3 : 4)", "(lf < 1 ? 3 : 4)"),
     "test_k_exact_reconstruction"),
    ("pyramid_base_inward", ("{{0,3,2,1},{0,1,4,-1}", "{{0,1,2,3},{0,1,4,-1}"),
     "test_geometry_closed_surfaces_and_volume"),
    ("pyramid_map_apex", ("dw[d] = P[4][d] - Q;", "dw[d] = P[4][d] - P[0][d];"),
     "test_face_quadrature_integrates_bilinear_exactly"),
    ("rank_test_per_column_only", ("|| !(nv > 1e-8 * sqrt(amax))", ""),
     "test_degenerate_pyramid_stencils_are_rejected"),
]

PY_MUTANTS = [
    # name, file under oracle/, (original text, planted mistake), pins that must catch it
    ("adam_bias_correction_dropped", "mlp.py", ("    mh = m / (1 - b1 ** t)\n", "    mh = m\n"),
     "test_adam_bias_correction_closed_forms"),
    ("adam_eps_inside_the_root", "mlp.py", ("np.sqrt(vh) + eps", "np.sqrt(vh + eps)"), "test_adam_bias_correction_closed_forms"),
    ("class_weights_swapped", "mlp.py", ("c = np.where(y > 0.5, w_pos, w_neg)\n    # -y", "c = np.where(y > 0.5, w_neg, w_pos)\n    # -y"),
     "test_gradient_matches_finite_differences"),
    ("bf16_truncates", "mlp.py", ("u = ((u + 0x7FFF + lsb) >> 16) << 16", "u = (u >> 16) << 16"),
     "test_bf16_rounding_is_nearest_even"),
    ("bf16_hidden_activation_not_rounded", "mlp.py",
     ("h1r = r(np.maximum(a1, 0.0)) if h1 is None", "h1r = np.maximum(a1, 0.0) if h1 is None"),
     "test_bf16_rounding_places_worked_example"),
    ("bias_gradient_from_the_rounded_dh2", "mlp.py", ('g["b2"] = f(dh2).sum(axis=0)', 'g["b2"] = f(dh2r).sum(axis=0)'),
     "test_bf16_rounding_places_worked_example"),
    ("label_linear_weights", "__init__.py", ("/ (self.params.lam_central + self.nd)", "/ (self.params.lam_central + self.nd + 1)"),
     "test_labels_vanish_on_a_uniform_flow_and_flag_a_step"),
    ("parameter_order_eps_alpha", "__init__.py", ("self.lam_central, self.eps, self.alpha,", "self.lam_central, self.alpha, self.eps,"),
     "test_cwenoz_weights_worked_example"),
]


@pytest.fixture(scope="module")
def workdir(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not found")
    return tmp_path_factory.mktemp("mutants")


def _run_c_mutant(mutant, workdir, threads):
    """Plant the mistake in a copy of the oracle's C source, compile it, and
    run the named pins against it; returns (completed process, error)."""
    name, (old, new), pins = mutant
    src = open(SRC).read()
    if src.count(old) != 1:
        return None, f"mutation site of {name} not unique"
    msrc = os.path.join(workdir, f"{name}.c")
    with open(msrc, "w") as f:
        f.write(src.replace(old, new))
    lib = os.path.join(workdir, f"{name}.so")
    cc = subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
                         "-std=c11", "-D_GNU_SOURCE", "-o", lib, msrc, "-lm"], capture_output=True, text=True)
    if cc.returncode:
        return None, f"{name} does not compile:\n{cc.stderr[-2000:]}"
    env = dict(os.environ, UCNS_ORACLE_LIB=lib, OMP_NUM_THREADS=str(threads))
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_mlp.py"), "-q", "-x", "-p", "no:cacheprovider",
                        "-k", pins], env=env, capture_output=True, text=True, timeout=600, cwd=ROOT)
    return r, None


@pytest.fixture(scope="module")
def c_results(workdir, request):
    """Every selected C mutant, built and checked concurrently (one child
    pytest per mutant, the cores shared out among them)."""
    wanted = {it.callspec.params["name"] for it in request.session.items
              if getattr(it, "originalname", "") == "test_pins_reject_the_mutant" and hasattr(it, "callspec")}
    todo = [m for m in MUTANTS if m[0] in wanted]
    cores = os.cpu_count() or 1
    workers = max(1, min(8, cores, len(todo)))
    with ThreadPoolExecutor(workers) as ex:
        done = ex.map(lambda m: _run_c_mutant(m, workdir, max(1, cores // workers)), todo)
        return {m[0]: res for m, res in zip(todo, done)}


@pytest.mark.parametrize("name,edit,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_the_mutant(name, edit, pins, c_results):
    r, err = c_results[name]
    assert err is None, err
    assert "passed" in r.stdout or "failed" in r.stdout, r.stdout + r.stderr  # the pins ran
    assert r.returncode != 0, f"mutant {name} survived {pins}:\n{r.stdout[-2000:]}"


def _run_python_pins(tree, fname, source, pins):
    """Copy the Python sources into tree with oracle/<fname> replaced by
    source, and run the named pins there (they import the copy)."""
    skip = shutil.ignore_patterns("_build", "_lib", "csrc", "__pycache__", "*.so")
    for d in ("oracle", "paper_2609_07387_gb300", "tests"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(tree, d), ignore=skip)
    with open(os.path.join(tree, "oracle", fname), "w") as f:
        f.write(source)
    tests = [os.path.join(tree, "tests", t) for t in ("test_oracle_mlp.py", "test_oracle_pins.py")]
    return subprocess.run([sys.executable, "-m", "pytest", *tests, "-q", "-p", "no:cacheprovider", "-k", pins],
                          capture_output=True, text=True, timeout=600, cwd=tree)


def test_python_pins_pass_on_an_unmodified_copy(workdir):
    pins = " or ".join(sorted({m[3] for m in PY_MUTANTS}))
    src = open(os.path.join(ROOT, "oracle", "mlp.py")).read()
    r = _run_python_pins(os.path.join(workdir, "tree_unmodified"), "mlp.py", src, pins)
    assert r.returncode == 0 and "failed" not in r.stdout, r.stdout + r.stderr


@pytest.mark.parametrize("name,fname,edit,pins", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_pins_reject_the_python_mutant(name, fname, edit, pins, workdir):
    src = open(os.path.join(ROOT, "oracle", fname)).read()
    old, new = edit
    assert src.count(old) == 1, f"mutation site of {name} not unique"
    r = _run_python_pins(os.path.join(workdir, f"tree_{name}"), fname, src.replace(old, new), pins)
    assert "passed" in r.stdout or "failed" in r.stdout, r.stdout + r.stderr  # the pins ran
    assert r.returncode != 0, f"mutant {name} survived {pins}:\n{r.stdout[-2000:]}"
