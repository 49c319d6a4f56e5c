"""Plant plausible mistakes in copies of the oracle's C source and check that
the pins in oracle_pins.py catch every one (CPU only).

Each mutant is compiled with the oracle's own flags and exercised in a child
process, so a mutant that crashes cannot take the test session down; a mutant
counts as caught only when a named check raises AssertionError.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lbm_oracle.c")
PINS = os.path.join(ROOT, "tests", "oracle_pins.py")

# (name, text in lbm_oracle.c, replacement). Each text occurs exactly once.
MUTANTS = [
    ("feq_quadratic_coeff", "4.5 * eu * eu", "4.0 * eu * eu"),
    ("feq_uu_sign", "- 1.5 * uu", "+ 1.5 * uu"),
    ("feq_linear_coeff", "1.0 + 3.0 * eu", "1.0 + 2.0 * eu"),
    ("feq_drop_rho", "weight(i) * rho * (1.0", "weight(i) * (1.0"),
    ("guo_sign", "3.0 * (eF - uF)", "3.0 * (eF + uF)"),
    ("guo_drop_quadratic", "+ 9.0 * eu * eF", "+ 0.0 * eu * eF"),
    ("guo_prefactor", "(1.0 - 1.0 / (2.0 * tau)) * weight(i)", "weight(i)"),
    ("velocity_half_force", "(j[a] + 0.5 * F[a]) / rho", "(j[a] + F[a]) / rho"),
    ("velocity_no_rho", "u_out[a] = (j[a] + 0.5 * F[a]) / rho;", "u_out[a] = (j[a] + 0.5 * F[a]);"),
    ("relax_times_tau", "(f[i] - feq[i]) / tau", "(f[i] - feq[i]) * tau"),
    ("moment_wrong_axis", "j[a] += f[i] * E[i][a];", "j[a] += f[i] * E[i][(a + 1) % 3];"),
    ("stream_backwards", "int xd = wrap(x + E[i][0], nx)", "int xd = wrap(x - E[i][0], nx)"),
    ("stream_swap_yz", "yd = wrap(y + E[i][1], ny),", "yd = wrap(y + E[i][2], ny),"),
    ("bounce_no_reverse", "nxt[opposite(i) * N + c] = fs[i] - moving;", "nxt[i * N + c] = fs[i] - moving;"),
    ("bounce_dropped", "nxt[opposite(i) * N + c] = fs[i] - moving;", ";"),
    ("weight_axis", "if (i <= 6) return 1.0 / 18.0;", "if (i <= 6) return 1.0 / 36.0;"),
    ("weight_split", "if (i <= 6)", "if (i <= 5)"),
    ("table_entry", "{1, -1, 0}, {-1, 1, 0}", "{-1, 1, 0}, {1, -1, 0}"),
    ("force_field_index", "out[a] = F[a * N + c];", "out[a] = F[a + 3 * c];"),
    ("round_floor", "nearbyint(v / q)", "floor(v / q)"),
    ("round_fp16_mantissa", "round_format(v, 10, -14, 65504.0)", "round_format(v, 11, -14, 65504.0)"),
    ("round_unshifted", "w + oracle_round(f[i * N + c] - w, fmt)", "oracle_round(f[i * N + c], fmt)"),
    ("init_rho_ignored", "if (rho0) rho = rho0[c];", ";"),
    ("moving_wall_sign", "nxt[opposite(i) * N + c] = fs[i] - moving;", "nxt[opposite(i) * N + c] = fs[i] + moving;"),
    ("moving_wall_factor", "moving = 6.0 * weight(i) *", "moving = 2.0 * weight(i) *"),
    ("moving_wall_cell", "if (u_wall && is_moving_wall(flags, d))", "if (u_wall && is_moving_wall(flags, c))"),
    ("inc_feq_rho_scaled", "weight(i) * (rho + 3.0 * cu", "weight(i) * rho * (1.0 + 3.0 * cu"),
    ("inc_feq_quadratic", "4.5 * cu * cu", "4.0 * cu * cu"),
    ("inc_velocity_over_rho", "u_out[a] = mom[a] + F[a] / 2.0;", "u_out[a] = (mom[a] + F[a] / 2.0) / r;"),
    ("inc_velocity_full_force", "u_out[a] = mom[a] + F[a] / 2.0;", "u_out[a] = mom[a] + F[a];"),
    ("inc_collide_ignores_model", "    if (model == 1) {\n        oracle_moments_incompressible(f, F, &rho, u);",
     "    if (model == 7) {\n        oracle_moments_incompressible(f, F, &rho, u);"),
    ("inc_init_ignores_model", "            if (model == 1)\n                oracle_equilibrium_incompressible",
     "            if (model == 7)\n                oracle_equilibrium_incompressible"),
    ("inc_step_ignores_model", "oracle_collide_cell_model(model, f, tau, Fc, fs);", "oracle_collide_cell_model(0, f, tau, Fc, fs);"),
    ("inc_sums_rho_weighted", "model == 1 ? uc[a] : r * uc[a]", "r * uc[a]"),
    ("split_whole_deviation", "double g = oracle_round((P[i] - w) - base, fmt);",
     "double g = oracle_round(P[i] - w, fmt) - base;"),
    ("split_base_sign", "double base = 3.0 * w * (E[i][0]", "double base = -3.0 * w * (E[i][0]"),
    ("split_store_no_bounce", "v[i] = is_fluid(flags, d) ? f[i * N + d] : f[opposite(i) * N + c];",
     "v[i] = f[i * N + d];"),
    ("split_rebuild_own_slot", "f[i * N + c] = is_fluid(flags, s) ? P[i * N + s] : P[opposite(i) * N + c];",
     "f[i * N + c] = is_fluid(flags, s) ? P[i * N + s] : P[i * N + c];"),
    ("split_step_unrounded", "if (is_split(fmt)) oracle_split_round(fs, fmt);", "if (0) oracle_split_round(fs, fmt);"),
]


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, (name, src.count(old))
    mpath = tmp_path / ("mut_%s.c" % name)
    mpath.write_text(src.replace(old, new))
    lib = tmp_path / ("libmut_%s.so" % name)
    subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math",
                           "-fopenmp", "-fPIC", "-shared", str(mpath), "-o", str(lib), "-lm"])
    return lib


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(tmp_path, name, old, new):
    lib = _build_mutant(tmp_path, name, old, new)
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, PINS, str(lib)], capture_output=True, text=True,
                       timeout=600, env=env)
    assert r.returncode == 1 and "FAILED_CHECK check_" in r.stdout, (name, r.returncode,
                                                                      r.stdout[-500:], r.stderr[-2000:])


def test_unmutated_source_passes_runner():
    r = subprocess.run([sys.executable, PINS, os.path.join(ROOT, "oracle", "liblbm_oracle.so")],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
