"""Planted-mistake (mutation) checks of the oracle's pins (CPU only).

Each mutant below is a copy of ``oracle/rt_oracle.c`` (or of the Python
half, ``oracle/oracle.py``) with ONE plausible mistake planted in it -- a dropped factor or term, a wrong sign, a transposed
operand or index, the wrong cross-section or Planck function -- and the pins
named beside it must fail on that build.  A mutant that every named pin
passes would be a mistake the oracle could carry unnoticed.  The unmodified
source, compiled the same way, must pass the union of the named pins (the
control).  The builds and pin runs go to subprocesses in parallel, each
loading its library through ``RT_ORACLE_LIB`` (and a planted oracle.py
through ``RT_ORACLE_PY``).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
SRC = os.path.join(ORACLE, "rt_oracle.c")

PRIM = "tests/test_oracle_primitives.py::"
PHYS = "tests/test_oracle_physics.py::"

# name: (text in rt_oracle.c, planted replacement, pins that must fail)
MUTANTS = {
    # Philox4x32-10 (published definition) and the uniform of a 64-bit word
    "philox_weyl_constant": ("k1 += 0xBB67AE85u;", "k1 += 0xBB67AE84u;",
                             [PRIM + "test_philox_matches_curand_host_generator"]),
    "philox_word_permutation": ("c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;",
                                "c0 = n0; c1 = lo0; c2 = n2; c3 = lo1;",
                                [PRIM + "test_philox_matches_curand_host_generator"]),
    "uniform_drops_a_bit": ("return (double)((w >> 11) + 1u) * 0x1p-53;",
                            "return (double)((w >> 12) + 1u) * 0x1p-53;",
                            [PRIM + "test_uniform_stream_statistics"]),
    # Planck function, dB/dT, Eq. 4
    "planck_drops_factor_2": ("return 2.0 * OR_H * nu * nu * nu / (OR_C * OR_C) / expm1(x);",
                              "return OR_H * nu * nu * nu / (OR_C * OR_C) / expm1(x);",
                              [PHYS + "test_planck_sum_matches_stefan_boltzmann"]),
    "dbdt_wrong_denominator": ("return pre * (x / T) / (expm1(x) * (-expm1(-x)));",
                               "return pre * (x / T) / (expm1(x) * expm1(x));",
                               [PHYS + "test_planck_peak_and_derivative"]),
    "eq4_drops_4pi": ("if (4.0 * OR_PI * or_planck_mean(m, s, mid) < target) lo = mid; else hi = mid;",
                      "if (OR_PI * or_planck_mean(m, s, mid) < target) lo = mid; else hi = mid;",
                      [PHYS + "test_temperature_solve_gray_closed_form"]),
    "eq4_drops_dnu": ("acc += m->kabs[s * m->nf + j] * or_planck_B(m->nu[j], T) * m->dnu[j];",
                      "acc += m->kabs[s * m->nf + j] * or_planck_B(m->nu[j], T);",
                      [PHYS + "test_temperature_solve_gray_closed_form"]),
    "eq4_cell_volume_h2": ("double rv = rho_of(m, s, c) * h[c] * h[c] * h[c];",
                           "double rv = rho_of(m, s, c) * h[c] * h[c];",
                           [PHYS + "test_optically_thin_equilibrium_temperature"]),
    "guess_4pi_for_16pi": ("q += r2 > 0.0 ? src[i].L / (16.0 * OR_PI * sigma * r2) : INFINITY;",
                           "q += r2 > 0.0 ? src[i].L / (4.0 * OR_PI * sigma * r2) : INFINITY;",
                           [PHYS + "test_temperature_guess_closed_form"]),
    # emission (Sect. 2, Eq. 1)
    "source_norm_drops_dnu": ("tot += lnu[j] * m->dnu[j];", "tot += lnu[j];",
                              [PHYS + "test_source_spectrum_is_the_normalised_blackbody"]),
    "iso_hemisphere": ("double mu = 1.0 - 2.0 * (1.0 - u2);", "double mu = 1.0 - (1.0 - u2);",
                       [PHYS + "test_empty_grid_emission_spectrum_and_isotropy"]),
    "iso_half_azimuth": ("double phi = 2.0 * OR_PI * (1.0 - u1);", "double phi = OR_PI * (1.0 - u1);",
                         [PHYS + "test_empty_grid_emission_spectrum_and_isotropy"]),
    "eq1_bin_left_edge": ("const double u = ((double)b + 0.5) / (double)p->source_bins;",
                          "const double u = (double)b / (double)p->source_bins;",
                          [PHYS + "test_equal_energy_source_bins"]),
    # Henyey-Greenstein (Eq. 15) and the direction rotation
    "hg_drops_square": ("mu = (1.0 + g * g - t * t) / (2.0 * g);",
                        "mu = (1.0 + g * g - t) / (2.0 * g);",
                        [PRIM + "test_hg_sampler_moments_and_ks"]),
    "rotate_transposed_operand": ("n[0] = st * (k[0] * k[2] * cp - k[1] * sp) / t + k[0] * mu;",
                                  "n[0] = st * (k[0] * k[2] * cp - k[1] * sp) / t + k[1] * mu;",
                                  [PRIM + "test_rotation_preserves_scattering_angle"]),
    "rotate_sign": ("n[2] = -st * cp * t + k[2] * mu;", "n[2] = st * cp * t + k[2] * mu;",
                    [PRIM + "test_rotation_preserves_scattering_angle"]),
    # cell traversal (uniform and refined)
    "dda_multiplies_by_k": ("if (k[a] > 0.0) t = (lo + h - x[a]) / k[a];",
                            "if (k[a] > 0.0) t = (lo + h - x[a]) * k[a];",
                            [PRIM + "test_dda_chords_match_brute_force"]),
    "dda_wrong_face": ("x[a] = step > 0 ? lo + h : lo;", "x[a] = step > 0 ? lo : lo + h;",
                       [PRIM + "test_dda_chords_match_brute_force"]),
    "refined_entry_sub_cube": ("p->s[a] = step > 0 ? 0 : m->refine - 1;", "p->s[a] = 0;",
                               [PRIM + "test_refined_dda_chords_match_brute_force"]),
    # flight, interaction and estimators (Sects. 2, 3.1, Eqs. 2-3)
    "extinction_drops_scattering": (
        "chi += rho_of(m, s, c) * (m->kabs[s * m->nf + j] + m->ksca[s * m->nf + j]);",
        "chi += rho_of(m, s, c) * m->kabs[s * m->nf + j];",
        [PHYS + "test_scattering_only_matches_brute_force_walk"]),
    "eq3_multiplies": ("double d = tau / chi;", "double d = tau * chi;",
                       [PHYS + "test_lucy_and_count_estimators_agree_per_species"]),
    "albedo_inverted": ("if (rng_u(&r) < albedo) {", "if (rng_u(&r) < 1.0 - albedo) {",
                        [PHYS + "test_scattering_only_matches_brute_force_walk"]),
    "lucy_full_chord_at_interaction": ("if (C->lucy[c]) lucy_deposit(C, o, c, j, d);",
                                       "if (C->lucy[c]) lucy_deposit(C, o, c, j, t);",
                                       [PHYS + "test_lucy_and_count_estimators_agree_per_species"]),
    "lucy_by_extinction": (
        "double ta = m->kabs[s * m->nf + j] * rho_of(m, s, c) * l;",
        "double ta = (m->kabs[s * m->nf + j] + m->ksca[s * m->nf + j]) * rho_of(m, s, c) * l;",
        [PHYS + "test_lucy_and_count_estimators_agree_per_species"]),
    "lucy_cells_count_absorptions_too": ("if (!C->lucy[c]) {\n            o->E_abs[s * nc + c] += C->xi;",
                                         "if (1) {\n            o->E_abs[s * nc + c] += C->xi;",
                                         [PHYS + "test_lucy_and_count_estimators_agree_per_species"]),
    "species_by_wrong_cross_section": (
        "w[s] = rho_of(m, s, c) * (sca ? m->ksca[s * m->nf + j] : m->kabs[s * m->nf + j]);",
        "w[s] = rho_of(m, s, c) * (sca ? m->kabs[s * m->nf + j] : m->ksca[s * m->nf + j]);",
        [PHYS + "test_lucy_and_count_estimators_agree_per_species"]),
    "escape_bin_wrong_axis": ("int b = (int)floor((k[2] + 1.0) * 5.0);",
                              "int b = (int)floor((k[0] + 1.0) * 5.0);",
                              [PHYS + "test_photon_counting_matches_escape_tallies"]),
    "lucy_criterion_inverted": ("C.lucy[c] = mx < p->lucy_tau;", "C.lucy[c] = mx > p->lucy_tau;",
                                [PHYS + "test_lucy_cells_are_those_below_the_face_to_face_threshold"]),
    "lucy_criterion_cell_diagonal": ("double t = chi_ext(m, c, j) * C.h[c];",
                                     "double t = chi_ext(m, c, j) * C.h[c] * sqrt(3.0);",
                                     [PHYS + "test_lucy_cells_are_those_below_the_face_to_face_threshold"]),
    "event_stores_outgoing_direction": (
        "e->k[0] = k[0]; e->k[1] = k[1]; e->k[2] = k[2];",
        "double kk[3] = { k[0], k[1], k[2] }; or_rotate(kk, mu, phi);"
        " e->k[0] = kk[0]; e->k[1] = kk[1]; e->k[2] = kk[2];",
        [PHYS + "test_stored_events_carry_the_incoming_direction"]),
    "mrw_sphere_reaches_past_the_far_face": ("double d1 = x[a] - lo, d2 = lo + h - x[a];",
                                             "double d1 = x[a] - lo, d2 = lo + 2.0 * h - x[a];",
                                             [PRIM + "test_refined_mrw_sphere_stays_in_the_sub_cube"]),
    "sub_cube_axes_swapped": ("p->s[0] = (int)(off % r);\n            p->s[1] = (int)((off / r) % r);",
                              "p->s[1] = (int)(off % r);\n            p->s[0] = (int)((off / r) % r);",
                              [PHYS + "test_pah_reemission_positions_and_directions"]),
    "source_drawn_uniformly": ("if (C->nsrc > 1) si = pick_cdf(C->src_L, C->nsrc, rng_u(&r));",
                               "if (C->nsrc > 1) si = (int)(rng_u(&r) * C->nsrc) % C->nsrc;",
                               [PHYS + "test_sources_emit_in_proportion_to_their_luminosity"]),
    "mrw_deposit_by_extinction": (
        "double e = C->xi * m->kabs[s * m->nf + j] * rho_of(m, s, c) * l;",
        "double e = C->xi * (m->kabs[s * m->nf + j] + m->ksca[s * m->nf + j]) * rho_of(m, s, c) * l;",
        [PHYS + "test_mrw_on_and_off_agree"]),
    "frozen_t_samples_dbdt": (": or_planck_B(m->nu[l], T);", ": or_planck_dBdT(m->nu[l], T);",
                              [PHYS + "test_bw_and_iterative_reach_the_same_temperatures"]),
    "eq4_bracket_not_widened": (
        "while (4.0 * OR_PI * or_planck_mean(m, s, hi) < target && hi < 1e12) hi *= 2.0;",
        "while (0) hi *= 2.0;",
        [PHYS + "test_temperature_solve_inverts_planck_mean"]),
    "guess_cap_raised": ("if (!(t < 2000.0)) t = 2000.0;", "if (!(t < 20000.0)) t = 20000.0;",
                         [PHYS + "test_temperature_guess_closed_form"]),
    "refined_cell_number_axes_reversed": ("return b + ((int64_t)p->s[2] * r + p->s[1]) * r + p->s[0];",
                                          "return b + ((int64_t)p->s[0] * r + p->s[1]) * r + p->s[2];",
                                          [PRIM + "test_refined_dda_chords_match_brute_force"]),
    "sub_cube_edge_not_divided": ("return p->f ? m->cell / m->refine : m->cell;", "return m->cell;",
                                  [PRIM + "test_refined_dda_chords_match_brute_force"]),
    "pc_y_from_the_x_axis": ("double yp = rel[0] * ey[0] + rel[1] * ey[1] + rel[2] * ey[2];",
                             "double yp = rel[0] * ex[0] + rel[1] * ex[1] + rel[2] * ex[2];",
                             [PHYS + "test_photon_counting_geometry_closed_forms"]),
    "camera_y_axis_flipped": ("ey[0] = -ct * cp; ey[1] = -ct * sp; ey[2] = st;",
                              "ey[0] = ct * cp; ey[1] = ct * sp; ey[2] = -st;",
                              [PHYS + "test_photon_counting_geometry_closed_forms"]),
    "pah_absorption_reemitted": ("\n        if (m->is_pah && m->is_pah[s]) {", "\n        if (0) {",
                                 [PHYS + "test_pah_packets_are_stored_and_counted"]),
    "eq4_bisection_stops_early": ("while (hi - lo > 1e-12 * hi) {", "while (hi - lo > 1e-4 * hi) {",
                                  [PHYS + "test_temperature_solve_inverts_planck_mean"]),
    "cdf_pick_one_bin_late": ("        if (acc >= target) return j;",
                              "        if (acc >= target) return j + (j < n - 1);",
                              [PHYS + "test_empty_grid_emission_spectrum_and_isotropy"]),
    "hg_isotropic_branch_half_range": ("        mu = 2.0 * z - 1.0;", "        mu = z;",
                                       [PRIM + "test_hg_sampler_moments_and_ks"]),
    "mrw_bisection_reversed": ("        if (or_mrw_survival(mid) > u) lo = mid; else hi = mid;",
                               "        if (or_mrw_survival(mid) > u) hi = mid; else lo = mid;",
                               [PRIM + "test_mrw_sampler_moments_and_ks"]),
    # re-emission (Eqs. 5, 10)
    "bw_samples_b_not_dbdt": ("? or_planck_dBdT(m->nu[l], T)", "? or_planck_B(m->nu[l], T)",
                              [PHYS + "test_bw_and_iterative_reach_the_same_temperatures"]),
    "bw_volume_of_doubled_edge": ("double rv = rho_of(m, s, c) * C->h[c] * C->h[c] * C->h[c];",
                                  "double rv = rho_of(m, s, c) * 8.0 * C->h[c] * C->h[c] * C->h[c];",
                          [PHYS + "test_bw_and_iterative_reach_the_same_temperatures"]),
    # modified random walk (Sect. 3.2)
    "mrw_series_sign": ("s += (n & 1) ? t : -t;", "s += t;",
                        [PRIM + "test_mrw_series_forms_agree"]),
    "mrw_image_series_exponent": ("double t = exp(-(mm + 0.5) * (mm + 0.5) / y);",
                                  "double t = exp(-(mm + 0.5) / y);",
                                  [PRIM + "test_mrw_series_forms_agree"]),
    "mrw_path_drops_3": ("double l = 3.0 * chi * R0 * R0 * y;", "double l = chi * R0 * R0 * y;",
                         [PHYS + "test_mrw_on_and_off_agree"]),
    "mrw_absorbs_by_extinction": ("if (rng_u(&r) < -expm1(-ca * l)) {",
                                  "if (rng_u(&r) < -expm1(-chi * l)) {",
                                  [PHYS + "test_mrw_on_and_off_agree"]),
    # the separate source grid of Eq. 1 (blackbody cumulative, model bin edges)
    "bb_series_bernoulli_sign": ("-691.0 / 2730.0", "691.0 / 2730.0",
                                 [PHYS + "test_separate_source_grid_has_equal_energy_bins"]),
    "bb_tail_power_of_k": ("6.0 * x / ((double)k * k * k)", "6.0 * x / ((double)k * k)",
                           [PHYS + "test_separate_source_grid_has_equal_energy_bins"]),
    "edges_arithmetic_mean": ("for (int j = 1; j < m->nf; ++j) e[j] = sqrt(m->nu[j - 1] * m->nu[j]);",
                              "for (int j = 1; j < m->nf; ++j) e[j] = 0.5 * (m->nu[j - 1] + m->nu[j]);",
                              [PHYS + "test_separate_source_grid_has_equal_energy_bins"]),
    # photon counting (Sect. 4)
    "pc_pixel_offset": ("double fx = floor(xp / pix + 0.5 * n), fy = floor(yp / pix + 0.5 * n);",
                        "double fx = floor(xp / pix + 0.5 * n), fy = floor(yp / pix);",
                        [PHYS + "test_photon_counting_geometry_closed_forms"]),
    "pc_cone_reversed": ("if (kd >= cam->cos_accept) {", "if (-kd >= cam->cos_accept) {",
                         [PHYS + "test_photon_counting_matches_escape_tallies"]),
    # PAH re-emission pass (Sect. 2.1, Eqs. 6-7)
    "pah_class_ignored": ("j = pick_cdf(C->eps_w + (size_t)n * m->nf, m->nf, rng_u(&r));",
                          "j = pick_cdf(C->eps_w, m->nf, rng_u(&r));",
                          [PHYS + "test_pah_reemission_frequency_law_per_class"]),
    "pah_law_drops_dnu": ("C.eps_w[(size_t)n * m->nf + j] = ps->eps[(size_t)n * m->nf + j] * m->dnu[j];",
                          "C.eps_w[(size_t)n * m->nf + j] = ps->eps[(size_t)n * m->nf + j];",
                          [PHYS + "test_pah_reemission_frequency_law_per_class"]),
    "pah_position_cell_corner": ("for (int a = 0; a < 3; ++a) x[a] = pos_lo(m, &idx, a) + rng_u(&r) * h;",
                                 "for (int a = 0; a < 3; ++a) x[a] = pos_lo(m, &idx, a) + rng_u(&r) * rng_u(&r) * h;",
                                 [PHYS + "test_pah_reemission_positions_and_directions"]),
    # ray tracer (Sect. 4, Eqs. 12-17) and its adjoint
    "hg_phase_exponent": ("return (1.0 - g * g) / (4.0 * OR_PI * d * sqrt(d));",
                          "return (1.0 - g * g) / (4.0 * OR_PI * d);",
                          [PHYS + "test_scattering_source_normalisation"]),
    "eq16_volume_h2": ("double vol = h[e->cell] * h[e->cell] * h[e->cell];",
                       "double vol = h[e->cell] * h[e->cell];",
                       [PHYS + "test_scattering_source_normalisation"]),
    "ray_drops_one_minus_exp": (
        "I += eta[cells[q] * nfi + f] * lens[q] * phi_f(dt) * exp(-tau);",
        "I += eta[cells[q] * nfi + f] * lens[q] * exp(-tau);",
        [PHYS + "test_raytrace_axis_view_of_uniform_cube"]),
    "ray_attenuates_own_cell_twice": (
        "I += eta[cells[q] * nfi + f] * lens[q] * phi_f(dt) * exp(-tau);",
        "I += eta[cells[q] * nfi + f] * lens[q] * phi_f(dt) * exp(-tau - dt);",
        [PHYS + "test_raytrace_axis_view_of_uniform_cube"]),
    "eq17_d_not_squared": ("sed[ci * nfi + f] += I * apix / (cam->D * cam->D);",
                           "sed[ci * nfi + f] += I * apix / cam->D;",
                           [PHYS + "test_raytrace_optically_thin_flux_and_star"]),
    "star_drops_4": ("sed[ci * nfi + f] += lnu[j] * exp(-tau) / (4.0 * OR_PI * cam->D * cam->D);",
                     "sed[ci * nfi + f] += lnu[j] * exp(-tau) / (OR_PI * cam->D * cam->D);",
                     [PHYS + "test_raytrace_optically_thin_flux_and_star"]),
    "pixel_corner_not_centre": ("double xp = (ix + 0.5 - 0.5 * cam->npix) * p;",
                                "double xp = (ix - 0.5 * cam->npix) * p;",
                                [PHYS + "test_raytrace_image_symmetry"]),
    "adjoint_sign_behind": ("- kext * l * behind;", "+ kext * l * behind;",
                            [PHYS + "test_adjoint_matches_central_differences"]),
    "adjoint_drops_a_length": ("+ e * l * l * kext * dphi_f(dt)) * att[q]",
                               "+ e * l * kext * dphi_f(dt)) * att[q]",
                               [PHYS + "test_adjoint_matches_central_differences"]),
    "adjoint_star_sign": ("dL_drho[s * nc + cells[q]] += -w * F * kext * lens[q];",
                          "dL_drho[s * nc + cells[q]] += w * F * kext * lens[q];",
                          [PHYS + "test_adjoint_matches_central_differences"]),
}


# Mistakes planted in the Python half of the oracle (oracle/oracle.py), run
# with the unmodified C library: name -> (text, replacement, pins)
PY = os.path.join(ORACLE, "oracle.py")
PY_MUTANTS = {
    "vis_pixel_corner_not_centre": ("a = (np.arange(npix) + 0.5 - 0.5 * npix) * pix / cam.D",
                                    "a = (np.arange(npix) - 0.5 * npix) * pix / cam.D",
                                    [PHYS + "test_visibility_definition_pins"]),
    "vis_u_and_v_swapped": ("ph = np.exp(-2j * np.pi * (u * a[None, :] + v * a[:, None]))",
                            "ph = np.exp(-2j * np.pi * (u * a[:, None] + v * a[None, :]))",
                            [PHYS + "test_visibility_definition_pins"]),
    "vis_phase_sign": ("ph = np.exp(-2j * np.pi * (u * a[None, :] + v * a[:, None]))",
                       "ph = np.exp(2j * np.pi * (u * a[None, :] + v * a[:, None]))",
                       [PHYS + "test_visibility_definition_pins"]),
    "vis_flux_over_d_not_d2": ("* pix * pix / (cam.D * cam.D)", "* pix * pix / cam.D",
                               [PHYS + "test_visibility_definition_pins"]),
}


def _compile(src_text: str, out: str) -> None:
    c = out[:-3] + ".c"
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
                    "-I", ORACLE, "-o", out, c, "-lm"], check=True, capture_output=True)


def _run_pins(lib: str, pins, py: str = "") -> subprocess.CompletedProcess:
    env = dict(os.environ, RT_ORACLE_LIB=lib, OMP_NUM_THREADS="2")
    if py:
        env["RT_ORACLE_PY"] = py
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider",
                           "-m", "not gpu", *pins], cwd=ROOT, env=env, capture_output=True,
                          text=True, timeout=900)


def _one(name, text, workdir):
    lib = os.path.join(workdir, f"{name}.so")
    if name == "_control":
        pins = sorted({p for _, _, ps in MUTANTS.values() for p in ps})
    else:
        old, new, pins = MUTANTS[name]
        text = text.replace(old, new)
    _compile(text, lib)
    r = _run_pins(lib, pins)
    return r.returncode, (r.stdout + r.stderr)[-3000:]


def _one_py(name, lib, workdir):
    """A planted mistake in oracle.py (or, for "_pycontrol", the unmodified
    file run the same way), with the unmodified C library."""
    text = open(PY).read()
    if name == "_pycontrol":
        pins = sorted({p for _, _, ps in PY_MUTANTS.values() for p in ps})
    else:
        old, new, pins = PY_MUTANTS[name]
        text = text.replace(old, new)
    py = os.path.join(workdir, f"{name}.py")
    with open(py, "w") as f:
        f.write(text)
    r = _run_pins(lib, pins, py)
    return r.returncode, (r.stdout + r.stderr)[-3000:]


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    text = open(SRC).read()
    for name, (old, _, _) in MUTANTS.items():
        assert text.count(old) == 1, f"mutant {name}: its site is not unique in rt_oracle.c"
    py_text = open(PY).read()
    for name, (old, _, _) in PY_MUTANTS.items():
        assert py_text.count(old) == 1, f"mutant {name}: its site is not unique in oracle.py"
    wd = str(tmp_path_factory.mktemp("oracle_mutants"))
    base = os.path.join(wd, "_unmodified.so")
    _compile(text, base)
    names = ["_control"] + list(MUTANTS)
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 2) as ex:
        futs = {n: ex.submit(_one, n, text, wd) for n in names}
        futs.update({n: ex.submit(_one_py, n, base, wd) for n in ["_pycontrol"] + list(PY_MUTANTS)})
        return {n: f.result() for n, f in futs.items()}


def test_unmodified_oracle_passes_every_named_pin(results):
    rc, log = results["_control"]
    assert rc == 0, log
    rc, log = results["_pycontrol"]
    assert rc == 0, log


@pytest.mark.parametrize("name", list(MUTANTS) + list(PY_MUTANTS))
def test_planted_mistake_fails_a_pin(results, name):
    rc, log = results[name]
    # pytest exits 1 when tests ran and some failed; a crash or a collection
    # error would not show that a pin caught the mistake
    assert rc == 1 and " failed" in log, f"mutant {name} survived its pins (rc {rc}):\n{log}"
