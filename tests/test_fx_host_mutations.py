"""The host check of the fixed-point operator's arithmetic catches plausible mistakes: each test
plants one mistake in a copy of paper_1905_11601_gb300/csrc/kv_fixed.cuh (a wrong wall weight, a
dropped cross product, a wrong neighbour, a wrong one-sided gap), builds tests/fx_host_check.cpp
against the copy, and requires the comparison with the oracle (tests/test_fx_host.py's bar) to
fail on at least one of a few cases. CPU only."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import Oracle
from paper_1905_11601_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
HDR = os.path.join(ROOT, "paper_1905_11601_gb300", "csrc", "kv_fixed.cuh")
TOL = 1e-10

MUTANTS = {
    "first_cell_weights": ("cls == 1 ? W3i{-8, 6, 2}", "cls == 1 ? W3i{-8, 5, 3}"),
    "cross_product_dropped": ("    M1 += (long long)a.l * b.h;\n", ""),
    "cross_part_not_shifted": ("((a.M1 + b.M1) >> FX_SPLIT)", "((a.M1 + b.M1) >> (FX_SPLIT + 1))"),
    "buoyancy_neighbour": ("b.mac(K.kb, fx_add(X(3, 0, 0, 0), X(3, 0, 0, 1)));",
                           "b.mac(K.kb, fx_add(X(3, 0, 0, 0), X(3, 0, 0, -1)));"),
    "upwind_wall_gap": ("if (back) return cls == 1 ? W3i{-12, 12, 0} : W3i{-6, 6, 0};",
                        "if (back) return W3i{-6, 6, 0};"),
    "upwind_face_direction": ("return back ? W3i{-24, 24, 0} : W3i{0, -24, 24};",
                              "return back ? W3i{0, -24, 24} : W3i{-24, 24, 0};"),
    "temperature_advecting_sum": ("a.mac(fx_mul(fx_add(B(0, -1, 0, 0), B(0, 0, 0, 0)), 2), fx_w3(d1x, txm, t0, txp));",
                                  "a.mac(fx_mul(fx_add(B(0, 0, 0, 0), B(0, 1, 0, 0)), 2), fx_w3(d1x, txm, t0, txp));"),
}

CASES = [(12, synth.CC, 1e6, 0, "auto", 0), (13, synth.AA, 3e6, 1, "general", 0), (11, synth.CC, 2e6, 0, "upwind", 1),
         (3, synth.AA, 1e6, 0, "upwind", 1)]


def worst_error(exe, tmp, n, bc, gr, tproj, mode, adv):
    pr = 0.71
    base = np.stack(synth.base_flow(n, n, n, bc, 31))
    o = Oracle(n, n, n, bc=bc, gr=gr, pr=pr, tproj=tproj, adv=adv)
    xp = o.project_input(synth.krylov_input(n, n, n, 32)[0])
    ref = o.jx_raw(base, xp)
    b, x, y = (str(tmp / f) for f in ("base.bin", "xp.bin", "y.bin"))
    base.tofile(b)
    xp.tofile(x)
    subprocess.check_call([exe, str(n), repr(gr), repr(pr), b, x, y, mode])
    out = np.fromfile(y).reshape(xp.shape)
    inner = (slice(1, n + 1),) * 3
    return max(np.abs(out[F][inner] - ref[F][inner]).max() / np.abs(ref[F][inner]).max() for F in range(4))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_the_host_check(name, tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    old, new = MUTANTS[name]
    src = open(HDR).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    inc = tmp_path / "inc"
    inc.mkdir()
    (inc / "kv_fixed.cuh").write_text(src.replace(old, new))
    exe = str(tmp_path / "fx_host_check_mut")
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-I", str(inc), os.path.join(HERE, "fx_host_check.cpp"), "-o", exe])
    errs = [worst_error(exe, tmp_path, *c) for c in CASES]
    assert max(errs) > TOL, (name, errs)
