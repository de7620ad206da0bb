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
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    import oracle
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"{name}: the text to mutate must occur exactly once"
    mutant_c = tmp_path / "mutant.c"
    mutant_c.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", *oracle.GCC_FLAGS, "-o", str(lib), str(mutant_c), "-lm", "-lpthread"])
    env = dict(os.environ, MFADVR_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", *PIN_FILES, "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"no pin caught the planted mistake '{name}':\n{r.stdout[-2000:]}"
