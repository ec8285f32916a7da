"""The fixed-point operator's arithmetic on the host, against the FP64 oracle (no GPU).

paper_1905_11601_gb300/csrc/kv_fixed.cuh holds the per-cell equations of the mixed path's
fixed-point operator as host-and-device code. tests/fx_host_check.cpp evaluates them at every
cell of a uniform cube with the grids the library chooses (base state and constants on one grid,
the projected input on its own), in both forms the GPU march uses (interior cells without the
first-derivative factor 3, and the wall-class weights everywhere). Here the result is compared
with the oracle's J P_BC x (Eqs (8)-(9) as used by Eqs (11)-(12)), per field, on random and on
smooth inputs (where the derivatives cancel most) and on cubes whose cells all touch a wall.
The GPU kernel itself is compared with the oracle in tests/test_gpu_variants.py.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import Oracle
from paper_1905_11601_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1905_11601_gb300", "csrc")
# per field: max |y_F - y_ref_F| <= TOL max |y_ref_F|; the mixed path's bar is 1e-9, the
# arithmetic carries about 2^-48 of the largest input and coefficient magnitudes
TOL = 1e-10


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("fx") / "fx_host_check")
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "fx_host_check.cpp"), "-o", exe])
    return exe


def run(driver, tmp, n, base, xp, gr, pr, mode):
    b, x, y = (str(tmp / f) for f in ("base.bin", "xp.bin", "y.bin"))
    np.ascontiguousarray(base, dtype=np.float64).tofile(b)
    np.ascontiguousarray(xp, dtype=np.float64).tofile(x)
    subprocess.check_call([driver, str(n), repr(gr), repr(pr), b, x, y, mode])
    return np.fromfile(y).reshape(xp.shape)


CASES = [(12, synth.CC, 1e6, 0, "random"), (13, synth.AA, 3e6, 0, "random"), (16, synth.AA, 3e6, 1, "smooth"),
         (9, synth.CC, 2e6, 0, "smooth"), (2, synth.CC, 1e6, 0, "random"), (3, synth.AA, 1e6, 1, "random")]


@pytest.mark.parametrize("n,bc,gr,tproj,kind", CASES)
@pytest.mark.parametrize("mode", ["auto", "general"])
def test_fixed_point_equations_match_oracle(driver, tmp_path, n, bc, gr, tproj, kind, mode):
    pr = 0.71
    base = np.stack(synth.base_flow(n, n, n, bc, 31))
    if kind == "random":
        x = synth.krylov_input(n, n, n, 32)[0]
    else:  # a smooth field: the derivatives cancel most of each term
        x = np.stack(synth.base_flow(n, n, n, bc, 33))
    o = Oracle(n, n, n, bc=bc, gr=gr, pr=pr, tproj=tproj)
    xp = o.project_input(x)
    ref = o.jx_raw(base, xp)
    y = run(driver, tmp_path, n, base, xp, gr, pr, mode)
    inner = (slice(1, n + 1),) * 3
    for F in range(4):
        r, g = ref[F][inner], y[F][inner]
        m = np.abs(r).max()
        assert m > 0
        assert np.abs(g - r).max() <= TOL * m, (F, np.abs(g - r).max() / m)


UPWIND_CASES = [(12, synth.CC, 1e6, 0, "random"), (13, synth.AA, 3e6, 1, "random"), (16, synth.AA, 3e6, 0, "smooth"),
                (2, synth.CC, 1e6, 0, "random"), (3, synth.AA, 1e6, 1, "smooth")]


@pytest.mark.parametrize("n,bc,gr,tproj,kind", UPWIND_CASES)
def test_fixed_point_upwind_equations_match_oracle(driver, tmp_path, n, bc, gr, tproj, kind):
    """The one-sided weights of the upwind reading (units of 1/(6h)), chosen per equation and axis
    by the FP64 base velocity, against the oracle's upwind branch."""
    pr = 0.71
    base = np.stack(synth.base_flow(n, n, n, bc, 31))
    x = synth.krylov_input(n, n, n, 32)[0] if kind == "random" else np.stack(synth.base_flow(n, n, n, bc, 33))
    o = Oracle(n, n, n, bc=bc, gr=gr, pr=pr, tproj=tproj, adv=1)
    xp = o.project_input(x)
    ref = o.jx_raw(base, xp)
    y = run(driver, tmp_path, n, base, xp, gr, pr, "upwind")
    inner = (slice(1, n + 1),) * 3
    for F in range(4):
        r, g = ref[F][inner], y[F][inner]
        m = np.abs(r).max()
        assert m > 0
        assert np.abs(g - r).max() <= TOL * m, (F, np.abs(g - r).max() / m)
    central = Oracle(n, n, n, bc=bc, gr=gr, pr=pr, tproj=tproj).jx_raw(base, xp)
    assert np.abs(central - ref).max() > 1e-6 * np.abs(ref).max()


_rng = np.random.default_rng(1905)
RANDOM_CASES = [(int(_rng.integers(2, 19)), int(_rng.integers(0, 2)), float(10 ** _rng.uniform(4, 7)),
                 int(_rng.integers(0, 2)), int(_rng.integers(0, 2)), int(_rng.integers(100, 10000)))
                for _ in range(8)]


@pytest.mark.parametrize("n,bc,gr,tproj,adv,seed", RANDOM_CASES)
def test_fixed_point_equations_on_seeded_random_cubes(driver, tmp_path, n, bc, gr, tproj, adv, seed):
    """Seeded random cube sizes, Grashof numbers, boundary types, projection readings and both
    advection schemes, with a base state scaled by a random power of ten (the grids follow it)."""
    pr = 0.71
    scale = 10.0 ** np.random.default_rng(seed).integers(-3, 4)
    base = np.stack(synth.base_flow(n, n, n, bc, seed)) * scale
    x = synth.krylov_input(n, n, n, seed + 1)[0]
    o = Oracle(n, n, n, bc=bc, gr=gr, pr=pr, tproj=tproj, adv=adv)
    xp = o.project_input(x)
    ref = o.jx_raw(base, xp)
    y = run(driver, tmp_path, n, base, xp, gr, pr, "upwind" if adv else "auto")
    inner = (slice(1, n + 1),) * 3
    for F in range(4):
        r, g = ref[F][inner], y[F][inner]
        m = np.abs(r).max()
        assert np.abs(g - r).max() <= TOL * m, (F, np.abs(g - r).max() / m)


def test_grid_conversion_is_exact_where_it_should_be(driver, tmp_path):
    """A base state and an input whose values are small integers times powers of two: their
    conversions to the fixed-point grids are exact and so is every integer sum and product, which
    leaves the constants' conversion (2^-49 of E) and the final conversion to FP64. The result
    then matches the oracle to within FP64 rounding of the terms."""
    n, gr, pr = 8, 1e6, 0.71
    rng = np.random.default_rng(5)
    base = np.zeros((4, n + 2, n + 2, n + 2))
    base[:3] = rng.integers(-8, 9, size=base[:3].shape) / 64.0
    base[3] = rng.integers(-8, 9, size=base[3].shape) / 16.0
    x = rng.integers(-16, 17, size=base.shape) / 32.0
    o = Oracle(n, n, n, bc=synth.CC, gr=gr, pr=pr)
    xp = o.project_input(x)
    ref = o.jx_raw(base, xp)
    y = run(driver, tmp_path, n, base, xp, gr, pr, "general")
    inner = (slice(1, n + 1),) * 3
    for F in range(4):
        r, g = ref[F][inner], y[F][inner]
        assert np.abs(g - r).max() <= 1e-13 * np.abs(r).max(), F
