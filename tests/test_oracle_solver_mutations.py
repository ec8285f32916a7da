"""The solver pins catch plausible mistakes: each test plants one mistake in a copy of
oracle/solvers.py (a sign in a Givens rotation or in the minimal-residual update, an index in
the back substitution or the BiCG residual update, the direction of the Newton update, the
Chebyshev recurrence's coefficient or shift, the enclosing ellipse's centre) and runs
tests/test_oracle_solvers.py against it in a fresh process; at least one pin must fail. CPU only."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "solvers.py")

MUTANTS = {
    "givens_sign": ("g[j], g[j + 1] = cs[j] * g[j], -sn[j] * g[j]", "g[j], g[j + 1] = cs[j] * g[j], sn[j] * g[j]"),
    "back_substitution_row": ("y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]",
                              "y[i] = (g[i] - np.dot(H[i + 1, i + 1:k], y[i + 1:k])) / H[i, i]"),
    "bicg_residual_index": ("rh[i] = rh[i] - alpha * uh[i + 1]", "rh[i] = rh[i] - alpha * uh[i]"),
    "mr_tau_sign": ("g1 = g1p - tau12 * g2", "g1 = g1p + tau12 * g2"),
    "newton_direction": ("S = S - d", "S = S + d"),
    "chebyshev_tau_update": ("tau_next = 1.0 / (2.0 * e - tau * c2)", "tau_next = 1.0 / (2.0 * e + tau * c2)"),
    "chebyshev_shift_sign": ("y_next = 2.0 * tau_next * (matvec(y) - d * y)", "y_next = 2.0 * tau_next * (matvec(y) + d * y)"),
    "ellipse_centre": ("d = 0.5 * (re.max() + re.min())", "d = 0.5 * (re.max() - re.min())"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_solver_mistake_fails_a_pin(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mutated = tmp_path / "solvers_mut.py"
    mutated.write_text(src.replace(old, new))
    env = dict(os.environ, KV_SOLVERS_PATH=str(mutated), OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_solvers.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"no pin caught the mutation {name}:\n{r.stdout[-2000:]}"
