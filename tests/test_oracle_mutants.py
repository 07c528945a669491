"""Plausible mistakes planted in a copy of the oracle must each fail a pin.

Every mutant is a one-token edit of oracle/oracle.c, compiled to a private
library; the pins named beside it run against that library and at least one
of them must fail.  This shows the pins would catch that class of mistake.
"""
import os
import subprocess

import pytest

import oracle
import oracle_pins as P

MUTANTS = [
    # (name, original text, replacement, pins expected to catch it)
    ("ode_sign_as_printed", "return 3.0 * M * u * u - u;", "return 3.0 * M * u * u + u;",
     [P.first_integral, P.straight_lines_m0]),
    ("gr_term_coefficient", "return 3.0 * M * u * u - u;", "return 2.0 * M * u * u - u;",
     [P.exit_angle, P.shadow_edge]),
    ("tableau_a41", "{44.0 / 45, -56.0 / 15", "{44.0 / 46, -56.0 / 15", [P.exit_angle]),
    ("fifth_order_weight", "-2187.0 / 6784, 11.0 / 84, 0}", "-2187.0 / 6784, 11.0 / 85, 0}",
     [P.exit_angle, P.first_integral]),
    ("embedded_weight", "393.0 / 640", "393.0 / 641", [P.step_order]),
    ("euclidean_v0", "pl->v0 = -pl->u0 * cot * sqrt(1.0 - 2.0 * M * pl->u0);",
     "pl->v0 = -pl->u0 * cot;", [P.shadow_edge, P.b_matches_v0]),
    ("b_without_redshift", "pl->b = r * pl->sin_a / sqrt(1.0 - 2.0 * M / r);",
     "pl->b = r * pl->sin_a;", [P.b_matches_v0]),
    ("hermite_basis", "double h4 = -4 * t3 + 7 * t4 - 3 * t5;",
     "double h4 = -4 * t3 + 7 * t4 - 2 * t5;", [P.exit_angle_render_tol, P.exit_angle]),
    ("disk_node_sign", "double p0 = atan2(-a, c);", "double p0 = atan2(a, c);", [P.disk_m0]),
    ("sphere_g_sign", "return 1.0 - 2.0 * u *", "return 1.0 + 2.0 * u *", [P.spheres_m0]),
    ("sky_parity", "base[(i + j) & 1]", "base[(i + j + 1) & 1]", [P.sky_cells]),
    ("map_back_transposed", "dirv[k] = cp * pl.e1[k] + sp * pl.e2[k];",
     "dirv[k] = sp * pl.e1[k] + cp * pl.e2[k];", [P.straight_lines_m0]),
    ("splitmix_constant", "0xBF58476D1CE4E5B9ull", "0xBF58476D1CE4E5B8ull", [P.splitmix_vector]),
    ("camera_rows_flipped", "double sy = (1.0 - 2.0 * (py + 0.5) / cam->h)",
     "double sy = (2.0 * (py + 0.5) / cam->h - 1.0)", [P.camera_convention]),
    ("camera_half_fov", "double th = tan(0.5 * cam->fov_deg", "double th = tan(0.55 * cam->fov_deg",
     [P.camera_convention]),
    ("capture_radius", "1.0 / (2.0 * M) : INFINITY", "1.0 / (4.0 * M) : INFINITY",
     [P.capture_iff_subcritical, P.hits_on_surfaces_m1]),
    ("disk_colour_inverted", "double t = pow(sc->disk_r_in / r, 0.75);",
     "double t = pow(r / sc->disk_r_in, 0.75);", [P.disk_colour_ends]),
    ("sphere_normal_sign", "double lam = 0.25 + 0.75 * fmax(0.0, -dot3(N, T));",
     "double lam = 0.25 + 0.75 * fmax(0.0, dot3(N, T));", [P.hits_on_surfaces_m1, P.spheres_m0]),
    # the paper's polyline method
    ("rk4_weight", "*u = u0 + h / 6.0 * (ku1 + 2.0 * ku2 + 2.0 * ku3 + ku4);",
     "*u = u0 + h / 6.0 * (ku1 + 2.0 * ku2 + 1.0 * ku3 + 2.0 * ku4);", [P.polyline_escape_order]),
    ("rk4_half_step", "double ku3 = v0 + 0.5 * h * kv2, kv3 = accel(M, u0 + 0.5 * h * ku2);",
     "double ku3 = v0 + 0.5 * h * kv2, kv3 = accel(M, u0 + h * ku2);", [P.polyline_escape_order]),
    ("escape_interpolation_end", "ev->phi_esc = phi + eps * u / (u - un);",
     "ev->phi_esc = phi + eps * un / (u - un);", [P.polyline_straight_m0, P.polyline_escape_order]),
    ("segment_plane_parameter", "double s = za / (za - zb), X[3];", "double s = zb / (za - zb), X[3];",
     [P.polyline_straight_m0, P.polyline_nodes]),
    # Keplerian disk shading
    ("kepler_newtonian_speed", "double beta = sqrt(M / (r - 2.0 * M));", "double beta = sqrt(M / r);",
     [P.doppler_closed_form]),
    ("doppler_direction_sign", "kin[k] = -(kr * xr_dir[k] + kt * t_dir[k]) / nk;",
     "kin[k] = (kr * xr_dir[k] + kt * t_dir[k]) / nk;", [P.doppler_closed_form]),
    # image sky
    ("sky_bilinear_weight", "rgb[c] = (1.0 - fy) * ((1.0 - fx) * c00 + fx * c10) + fy * ((1.0 - fx) * c01 + fx * c11);",
     "rgb[c] = (1.0 - fy) * (fx * c00 + (1.0 - fx) * c10) + fy * ((1.0 - fx) * c01 + fx * c11);",
     [P.sky_texture_affine]),
    ("sky_texel_centre", "double x = phi / (2.0 * OR_PI) * W - 0.5, y = theta / OR_PI * H - 0.5;",
     "double x = phi / (2.0 * OR_PI) * W, y = theta / OR_PI * H - 0.5;", [P.sky_texture_affine]),
    # anti-aliased pixels
    ("spp_grid_offset", "double sx = x + (i + 0.5) / n - 0.5, sy = y + (j + 0.5) / n - 0.5;",
     "double sx = x + (i + 0.0) / n - 0.5, sy = y + (j + 0.0) / n - 0.5;", [P.spp_mean]),
]


@pytest.fixture(scope="module")
def src():
    with open(oracle.SRC) as f:
        return f.read()


@pytest.mark.parametrize("name,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, src, name, old, new, pins):
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mutated = src.replace(old, new, 1)
    c = tmp_path / f"{name}.c"
    c.write_text(mutated)
    so = str(tmp_path / f"{name}.so")
    oracle.build(out=so, src=str(c), openmp=False)
    lib = oracle.load(so)
    results = []
    for pin in pins:
        try:
            ok, detail = pin(lib)
        except Exception as e:  # a crash in the pin counts as caught
            ok, detail = False, f"raised {type(e).__name__}: {e}"
        results.append((pin.__name__, ok, detail))
    assert any(not ok for _, ok, _ in results), f"{name} survived: {results}"
