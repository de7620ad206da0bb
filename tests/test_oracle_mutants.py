"""The oracle's pins catch plausible mistakes in it.

Each case plants one mistake in a copy of oracle/mfa_oracle.c (a wrong knot,
index, sign, factor, operand or order of operations, in the basis, the
queries, the Hessian or the ray caster), compiles the copy, and runs the
oracle's pin tests against it in a subprocess: at least one pin must fail.
The mistakes live only in those throwaway copies, on the CPU."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mfa_oracle.c")
PIN_FILES = ["tests/test_oracle_pins.py", "tests/test_oracle_knots.py", "tests/test_oracle_nurbs.py",
             "tests/test_oracle_hessian.py"]

# name: (text in the oracle, planted replacement)
MUTANTS = {
    "interior_knots": ("t[p + j] = (double)j / (double)m;", "t[p + j] = (double)j / (double)(m + 1);"),
    "span_tie_left": ("if (u < t[mid]) hi = mid;", "if (u <= t[mid]) hi = mid;"),
    "recurrence_denominator": ("val += (u - t[i]) / (t[i + q] - t[i]) * B[q - 1][r - 1];",
                               "val += (u - t[i]) / (t[i + q + 1] - t[i]) * B[q - 1][r - 1];"),
    "derivative_sign": ("if (r < p) d -= (double)p / (t[i + p + 1] - t[i + 1]) * B[p - 1][r];",
                        "if (r < p) d += (double)p / (t[i + p + 1] - t[i + 1]) * B[p - 1][r];"),
    "derivative_factor": ("if (r > 0) d += (double)p / (t[i + p] - t[i]) * B[p - 1][r - 1];",
                          "if (r > 0) d += (double)(p + 1) / (t[i + p] - t[i]) * B[p - 1][r - 1];"),
    "gradient_axis_transposed": ("fv += N[0][a] * dN[1][b] * N[2][c2] * P;",
                                 "fv += dN[0][a] * N[1][b] * N[2][c2] * P;"),
    "rational_quotient_sign": ("out[d] = (h[d] - f * g[d]) / g[0];", "out[d] = (h[d] + f * g[d]) / g[0];"),
    "brute_endpoint": ("if (u >= t[n] && i == n - 1) return 1.0;", "if (u > t[n] && i == n - 1) return 1.0;"),
    "brute_dk_sign": ("if (d2 > 0.0) v -= (double)p / d2 * orc_basis_brute_dk(",
                      "if (d2 > 0.0) v += (double)p / d2 * orc_basis_brute_dk("),
    "hessian_dropped_term": ("(h[4 + o] - f1[di] * g[1 + dj] - f1[dj] * g[1 + di] - f * g[4 + o]) / W;",
                             "(h[4 + o] - f1[di] * g[1 + dj] - f * g[4 + o]) / W;"),
    "hessian_cross_orders_swapped": ("{0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};",
                                     "{0, 2, 0}, {0, 0, 2}, {1, 0, 1}, {1, 1, 0}, {0, 1, 1}};"),
    "tf_interpolation_reversed": ("rgba[c] = a + fr * (b - a);", "rgba[c] = b + fr * (a - b);"),
    "sample_placement": ("double t = t0 + ((double)k + 0.5) * rp->step;",
                         "double t = t0 + ((double)k + 0.25) * rp->step;"),
    "opacity_exponent_inverted": ("alpha = 1.0 - pow(1.0 - alpha, ratio);",
                                  "alpha = 1.0 - pow(1.0 - alpha, 1.0 / ratio);"),
    "compositing_weight": ("double w = (1.0 - A) * alpha;", "double w = alpha;"),
    "shading_ka_kd_swapped": ("rgba[c] = clamp01(rgba[c] * (rp->ka + rp->kd * ndl) + rp->ks * spec);",
                              "rgba[c] = clamp01(rgba[c] * (rp->kd + rp->ka * ndl) + rp->ks * spec);"),
    "world_gradient_scale": ("double g[3] = {f[1] / ext[0], f[2] / ext[1], f[3] / ext[2]};",
                             "double g[3] = {f[1] * ext[0], f[2] / ext[1], f[3] / ext[2]};"),
    "fov_full_angle": ("double th = tan(cam->fovy_deg * (M_PI / 180.0) * 0.5);",
                       "double th = tan(cam->fovy_deg * (M_PI / 180.0));"),
    "rows_bottom_up": ("double sy = (1.0 - 2.0 * (y + 0.5) / H) * th;",
                       "double sy = (2.0 * (y + 0.5) / H - 1.0) * th;"),
    "slab_enter_not_advanced": ("if (ta > a0) { a0 = ta; b0 = ea; }", "if (ta < a0) { a0 = ta; b0 = ea; }"),
    "recurrence_right_denominator": ("val += (t[i + q + 1] - u) / (t[i + q + 1] - t[i + 1]) * B[q - 1][r];",
                                     "val += (t[i + q + 1] - u) / (t[i + q] - t[i + 1]) * B[q - 1][r];"),
    "lattice_index_transposed": (
        "return m->ctrl[(size_t)i + (size_t)m->n[0] * ((size_t)j + (size_t)m->n[1] * (size_t)k)];",
        "return m->ctrl[(size_t)j + (size_t)m->n[1] * ((size_t)i + (size_t)m->n[0] * (size_t)k)];"),
    "rational_numerator_unweighted": ("const double w = weight_at(m, i, j, k), wP = w * ctrl_at(m, i, j, k);",
                                      "const double w = weight_at(m, i, j, k), wP = ctrl_at(m, i, j, k);"),
    "knot_right_end_unchecked": ("if (t[i] != 0.0 || t[n + i] != 1.0) return -1;", "if (t[i] != 0.0) return -1;"),
    "zero_weight_accepted": ("if (!(m->weights[i] > 0.0) || !isfinite(m->weights[i])) return -1;",
                             "if (!(m->weights[i] >= 0.0) || !isfinite(m->weights[i])) return -1;"),
    "camera_right_flipped": ("cross3(cam->up, J.fwd, J.right);", "cross3(J.fwd, cam->up, J.right);"),
    "ortho_aspect_dropped": ("double sx = ((x + 0.5) / W - 0.5) * cam->ortho_height * aspect;",
                             "double sx = ((x + 0.5) / W - 0.5) * cam->ortho_height;"),
    "ortho_rows_bottom_up": ("double sy = (0.5 - (y + 0.5) / H) * cam->ortho_height;",
                             "double sy = ((y + 0.5) / H - 0.5) * cam->ortho_height;"),
    "perspective_direction_unnormalised": ("d[a] /= l;", "(void)l;"),
    "parallel_ray_high_side_kept": ("if (o[a] < m->box_min[a] || o[a] > m->box_max[a]) return 0;",
                                    "if (o[a] < m->box_min[a]) return 0;"),
    "sample_count_rounded_up": ("long N = (long)floor(r);", "long N = (long)ceil(r);"),
    "tf_range_offset_dropped": ("clamp01((v - J->lo) / (J->hi - J->lo))", "clamp01(v / (J->hi - J->lo))"),
    "tf_nearest_entry": ("double fr = x - i;", "double fr = floor(x - i + 0.5);"),
    "opacity_accumulates_alpha": ("A += w;", "A += alpha;"),
    "termination_not_strict": ("if (stop < 0 && A > rp->max_opacity) {", "if (stop < 0 && A >= rp->max_opacity) {"),
    "shading_one_sided": ("double ndl = fabs(-(g[0] * d[0] + g[1] * d[1] + g[2] * d[2]) / gn);",
                          "double ndl = fmax(0.0, -(g[0] * d[0] + g[1] * d[1] + g[2] * d[2]) / gn);"),
    "flat_field_diffuse": ("for (int c = 0; c < 3; ++c) rgba[c] *= rp->ka;",
                           "for (int c = 0; c < 3; ++c) rgba[c] *= rp->kd;"),
    "flat_threshold_strict": ("if (gn <= J->gthresh) {", "if (gn < J->gthresh) {"),
    "point_span_output_shifted": ("if (s3) s3[d] = s[d];", "if (s3) s3[d] = s[d] - 1;"),
    "point_clamp_dropped": ("for (int d = 0; d < 3; ++d) q[d] = clamp01((double)j->uvw[3 * i + d]);",
                            "for (int d = 0; d < 3; ++d) q[d] = (double)j->uvw[3 * i + d];"),
    "point_chunks_skip_first": ("jobs[t].begin = npts * t / nthreads;",
                                "jobs[t].begin = npts * t / nthreads + (t > 0);"),
    "render_rows_dealt_inverted": ("if ((rows_done++ % J->nthreads) != ra->tid) continue;",
                                   "if ((rows_done++ % J->nthreads) == ra->tid) continue;"),
    "render_row_step_ignored": ("for (int y = 0; y < H; y += J->row_step) {", "for (int y = 0; y < H; y += 1) {"),
    "sample_count_tie_never_flagged": ("if (rn >= 1.0 && fabs(r - rn) < window) {",
                                       "if (rn >= 1.0 && fabs(r - rn) < 0.0) {"),
    "termination_tie_low_edge_dropped": ("if (lo < 0 && A > rp->max_opacity - ORC_TIE_OPACITY) lo = k + 1;",
                                         "if (lo < 0 && A > rp->max_opacity) lo = k + 1;"),
    "termination_tie_high_edge_dropped": ("if (A > rp->max_opacity + ORC_TIE_OPACITY) { hi = k + 1; break; }",
                                          "if (A > rp->max_opacity) { hi = k + 1; break; }"),
}


def _run_mutant(name, src, workdir):
    """Compile one mutant and run the pins against it: (exit code, output)."""
    import oracle
    old, new = MUTANTS[name]
    if src.count(old) != 1:
        return None, f"the text to mutate occurs {src.count(old)} times"
    mutant_c = os.path.join(workdir, f"{name}.c")
    with open(mutant_c, "w") as fh:
        fh.write(src.replace(old, new))
    lib = os.path.join(workdir, f"lib{name}.so")
    subprocess.check_call(["gcc", *oracle.GCC_FLAGS, "-o", lib, mutant_c, "-lm", "-lpthread"])
    env = dict(os.environ, MFADVR_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", *PIN_FILES, "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def mutant_results(tmp_path_factory):
    """Every mutant's pin run, several at a time (each is its own process)."""
    from concurrent.futures import ThreadPoolExecutor
    src = open(SRC).read()
    workdir = str(tmp_path_factory.mktemp("mutants"))
    names = sorted(MUTANTS)
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        return dict(zip(names, ex.map(lambda n: _run_mutant(n, src, workdir), names)))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, mutant_results):
    rc, out = mutant_results[name]
    assert rc is not None, f"{name}: {out}"
    assert rc != 0, f"no pin caught the planted mistake '{name}':\n{out}"
