"""The pins catch plausible mistakes: each test plants one mistake in a copy of the oracle's C
source (a wrong index, a swapped weight, a dropped term, a wrong sign), builds it, and runs the
oracle pins against it in a fresh process; at least one pin must fail. CPU only."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "kv_oracle.c")

MUTANTS = {
    "interp_offset": ("for (int dc = -1; dc <= 0; ++dc)", "for (int dc = 0; dc <= 1; ++dc)"),
    "nonuniform_weights_swapped": ("return (dm * dm * (fp - f0) + dp * dp * (f0 - fm))",
                                   "return (dp * dp * (fp - f0) + dm * dm * (f0 - fm))"),
    "buoyancy_neighbour": ("if (F == FW) r += 0.5 * (at(c, xT, i, j, k) + at(c, xT, i, j, k + 1));",
                           "if (F == FW) r += 0.5 * (at(c, xT, i, j, k) + at(c, xT, i, j, k - 1));"),
    "eigenvalue_not_squared": ("c->lamp[a][m] = -4.0 / (h * h) * s * s;", "c->lamp[a][m] = -4.0 / (h * h) * s;"),
    "wall_pair_not_averaged": ("*lo0 = *lo1 = ml;", "*lo0 = ml;"),
    "advection_sign": ("-\n        advect_sel(c, xv, Ub, Th, FT, i, j, k);", "+\n        advect_sel(c, xv, Ub, Th, FT, i, j, k);"),
    "gradient_direction": ("double g = (phi[cidx(c, u[0], u[1], u[2])] - phi[cidx(c, t[0], t[1], t[2])]) /",
                           "double g = (phi[cidx(c, t[0], t[1], t[2])] - phi[cidx(c, u[0], u[1], u[2])]) /"),
    "wall_half_spacing_dropped": ("if (t <= 0) return 0.0;", "if (t <= 0) return -0.5 / n;"),
}

# Mistakes that only a stretched grid (Eq 22) can show; run against the stretched-grid pins.
STRETCH_MUTANTS = {
    "stretch_sign": ("c->xf[a][t] = xi - g->stretch * sin(2.0 * M_PI * xi);",
                     "c->xf[a][t] = xi + g->stretch * sin(2.0 * M_PI * xi);"),
    "stretch_centres_unmapped": ("for (int t = 1; t <= n; ++t) c->xc[a][t] = 0.5 * (c->xf[a][t - 1] + c->xf[a][t]);",
                                 "for (int t = 1; t <= n; ++t) c->xc[a][t] = ((double)t - 0.5) / n;"),
    "stretch_face_volume_is_cell_width": ("return face_like(F, a) ? centre_gap(c, a, t) : cell_width(c, a, t);",
                                          "return cell_width(c, a, t);"),
    "stretch_gradient_uses_cell_width": ("/ centre_gap(c, F, tf[F]);", "/ cell_width(c, F, tf[F]);"),
    "stretch_divergence_uses_centre_gap": ("/ cell_width(c, 0, i) +", "/ centre_gap(c, 0, i) +"),
    "stretch_one_sided_symmetrisation": ("S[(size_t)(t - 1) * n + t] = 1.0 / (g * sqrt(dx * cell_width(c, a, t + 1)));",
                                         "S[(size_t)(t - 1) * n + t] = 1.0 / (g * dx);"),
    "stretch_eigenvector_scaling_inverted": ("Q[(size_t)t * n + order[m]] / sqrt(cell_width(c, a, t + 1));",
                                             "Q[(size_t)t * n + order[m]] * sqrt(cell_width(c, a, t + 1));"),
}

# Mistakes in the optional upwind advection; run against its pins.
UPWIND_MUTANTS = {
    "upwind_selector_flipped": ("interp(c, sel[comp], comp, F, i, j, k) >= 0.0", "interp(c, sel[comp], comp, F, i, j, k) < 0.0"),
    "upwind_selected_by_perturbation": ("advect_sel(c, xv, Ub, Ub[F], F, i, j, k)", "advect_sel(c, xv, xv, Ub[F], F, i, j, k)"),
    "upwind_wall_gap_uniform": ("/ (x0 - coord(c, F, a, t[a] - 1));", "/ c->h[a];"),
    "upwind_forward_side_swapped": ("return (nb(c, f, i, j, k, a, +1) - f0) / (coord(c, F, a, t[a] + 1) - x0);",
                                    "return (f0 - nb(c, f, i, j, k, a, -1)) / (coord(c, F, a, t[a] + 1) - x0);"),
}

CASES = {name: (old, new, "test_oracle_pins.py") for name, (old, new) in MUTANTS.items()}
CASES.update({name: (old, new, "test_oracle_upwind.py") for name, (old, new) in UPWIND_MUTANTS.items()})
CASES.update({name: (old, new, "test_oracle_stretch.py") for name, (old, new) in STRETCH_MUTANTS.items()})


@pytest.mark.parametrize("name", sorted(CASES))
def test_planted_mistake_fails_a_pin(name, tmp_path):
    old, new, pins = CASES[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mutated = tmp_path / "kv_oracle_mut.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "libkv_oracle_mut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-D_DEFAULT_SOURCE",
                           "-o", str(lib), str(mutated), "-lm"])
    env = dict(os.environ, KV_ORACLE_LIB=str(lib), OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", pins)],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"no pin caught the mutation {name}:\n{r.stdout[-2000:]}"
