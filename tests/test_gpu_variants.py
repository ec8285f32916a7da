"""GPU parity of every compiled operator variant, the literal SIMPLE loop, non-finite inputs, the
device-side SIMPLE test and the layout/base-flow calls of the C ABI.

The autotuner picks one operator variant per grid by timing, so the other parity tests cover
whichever variant won on the box. Here kv_set_tuning pins each variant in turn (every FP64
block shape the tuner tries; every double-float candidate: the split pass at each block shape
and the 2.5D march at 16, 32 and 64 planes per block) and each is compared with the FP64 oracle
at ragged sizes that span several tiles and a tail.

Tolerances, per result: relative 2-norm over (u, v, w, T) and, per field F,
max |y_F - y_ref_F| <= tol * max |y_ref_F|, with tol = 1e-12 for the FP64 path and 1e-9 for the
mixed path (the spec bars)."""
import ctypes

import numpy as np
import pytest

from oracle import Oracle
from paper_1905_11601_gb300 import synth

pytestmark = pytest.mark.gpu
TOL64, TOLMIX = 1e-12, 1e-9
torch = pytest.importorskip("torch")

FP64_BLOCKS = [(32, 8), (64, 4), (128, 2), (32, 4), (16, 16), (256, 1)]
DF_VARIANTS = [(0, 32, 1), (0, 32, 2), (0, 64, 1), (0, 32, 4), (0, 64, 2), (0, 128, 1), (1, 0, 16), (1, 0, 32),
               (1, 0, 64), (2, 0, 8), (2, 0, 16), (2, 0, 32), (2, 0, 64)]
CASES = [((70, 65, 67), synth.CC, 2e6, 0), ((33, 18, 20), synth.AA, 3e6, 0), ((33, 18, 20), synth.AA, 3e6, 1),
         ((9, 130, 12), synth.AA, 3e6, 1)]
# the fixed-point operator (variant 2) serves cubic grids: ragged cubes against the tiles
CUBES = [((37, 37, 37), synth.CC, 2e6, 0), ((33, 33, 33), synth.AA, 3e6, 1), ((20, 20, 20), synth.AA, 3e6, 0),
         ((2, 2, 2), synth.CC, 1e6, 0), ((3, 3, 3), synth.AA, 1e6, 1)]  # every cell next to a wall


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_11601_gb300 import build
    build.build()


def kvmod():
    from paper_1905_11601_gb300 import kv
    return kv


_REF = {}


def reference(n, bc, gr, tproj, seed=41):
    """(base, x, y_ref) for a case; the oracle runs once per case."""
    key = (n, bc, gr, tproj, seed)
    if key not in _REF:
        base = np.stack(synth.base_flow(*n, bc, seed))
        x = synth.krylov_input(*n, seed + 1)[0]
        y_ref = Oracle(*n, bc=bc, gr=gr, pr=0.71, tproj=tproj).krylov_vector(base, x)
        _REF[key] = (base, x, y_ref)
    return _REF[key]


def check(y, y_ref, tol, label):
    rel = np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref)
    assert rel < tol, (label, "2-norm", rel)
    for F in range(4):
        m = np.abs(y_ref[F]).max()
        if m == 0:
            assert np.abs(y[F]).max() == 0, (label, F)
            continue
        e = np.abs(y[F] - y_ref[F]).max() / m
        assert e <= tol, (label, "field", F, e)


@pytest.mark.parametrize("n,bc,gr,tproj", CASES)
def test_every_fp64_block_shape_matches_oracle(n, bc, gr, tproj):
    kv = kvmod()
    base, x, y_ref = reference(n, bc, gr, tproj)
    g = kv.Grid(*n, bc=bc, gr=gr, pr=0.71, tproj=tproj)
    g.set_tuning(apply_block=FP64_BLOCKS[0])  # pinned before the base flow: no autotuning
    g.set_base_flow(torch.from_numpy(base).cuda())
    xt = torch.from_numpy(x).cuda()
    for blk in FP64_BLOCKS:
        g.set_tuning(apply_block=blk)
        assert g.tuning()["apply_block"] == blk
        check(g.krylov_vector(xt).cpu().numpy(), y_ref, TOL64, blk)


@pytest.mark.parametrize("n,bc,gr,tproj", CASES + CUBES + [((128, 128, 128), synth.AA, 3e6, 0)])
def test_every_double_float_variant_matches_oracle(n, bc, gr, tproj):
    kv = kvmod()
    base, x, y_ref = reference(n, bc, gr, tproj)
    g = kv.Grid(*n, bc=bc, gr=gr, pr=0.71, tproj=tproj, precision=kv.KV_PREC_MIXED)
    g.set_tuning(apply_block=(32, 8), df_variant=1, df_block=(0, 32))
    g.set_base_flow(torch.from_numpy(base).cuda())
    xt = torch.from_numpy(x).cuda()
    cubic = n[0] == n[1] == n[2]
    for v, bx, by in DF_VARIANTS:
        if v == 2 and not cubic:
            with pytest.raises(kv.KvError):
                g.set_tuning(apply_block=(32, 8), df_variant=v, df_block=(bx, by))
            continue
        g.set_tuning(apply_block=(32, 8), df_variant=v, df_block=(bx, by))
        t = g.tuning()
        assert t["df_variant"] == v and t["df_block"][1] == by
        y, st = g.krylov_vector(xt, stats=True)
        assert st.device_error == 0
        check(y.cpu().numpy(), y_ref, TOLMIX, (v, bx, by))


def test_mixed_256_matches_the_oracle_directly():
    """The benchmark workload (256^3 CC at the paper's critical Grashof number) in mixed
    precision, with the variant the autotuner picks, against the FP64 oracle itself."""
    kv = kvmod()
    w = synth.WORKLOADS["cube256_cc"]
    n = (w.nx, w.ny, w.nz)
    base, x = synth.workload_arrays(w)
    base = np.stack(base)
    g = kv.Grid(*n, bc=w.bc, gr=w.gr, pr=w.pr, precision=kv.KV_PREC_MIXED)
    g.set_base_flow(torch.from_numpy(base).cuda())
    y, st = g.krylov_vector(torch.from_numpy(x[0]).cuda(), stats=True)
    assert st.device_error == 0
    y = y.cpu().numpy()
    del g
    y_ref = Oracle(*n, bc=w.bc, gr=w.gr, pr=w.pr).krylov_vector(base, x[0])
    check(y, y_ref, TOLMIX, "256^3 mixed")


@pytest.mark.parametrize("prec", [0, 1])
def test_literal_simple_loop(prec):
    """Section 3.1's loop taken literally: with a tolerance no pass can meet, max_passes = 3
    passes run, the velocity stays the one-pass result (the later passes project a field that
    is already divergence-free), the pressure is the sum of the three corrections, and the call
    reports KV_ERR_NOT_CONVERGED."""
    kv = kvmod()
    n, bc, gr = (20, 14, 17), synth.AA, 2e6
    base = np.stack(synth.base_flow(*n, bc, 51))
    x = synth.krylov_input(*n, 52)[0]
    tol_bar = TOL64 if prec == 0 else TOLMIX
    g1 = kv.Grid(*n, bc=bc, gr=gr, precision=prec)
    g1.set_base_flow(torch.from_numpy(base).cuda())
    y1 = g1.krylov_vector(torch.from_numpy(x).cuda()).cpu().numpy()
    g3 = kv.Grid(*n, bc=bc, gr=gr, precision=prec, tol=1e-300, max_passes=3)
    g3.set_base_flow(torch.from_numpy(base).cuda())
    xt = torch.from_numpy(x).cuda()
    y3 = torch.full_like(xt, float("nan"))
    p3 = g3.empty()
    st = kv.Stats()
    rc = g3.lib.kv_krylov_vector(g3.h, xt.data_ptr(), y3.data_ptr(), p3.data_ptr(), ctypes.byref(st))
    assert rc == -3, g3.lib.kv_last_error(g3.h)  # KV_ERR_NOT_CONVERGED
    assert st.passes == 3
    assert b"max_passes" in g3.lib.kv_last_error(g3.h)
    y3 = y3.cpu().numpy()
    check(y3, y1, tol_bar, "velocity after 3 passes vs 1")
    o = Oracle(*n, bc=bc, gr=gr, tol=1e-300, max_passes=3)
    y_ref, p_ref, ost = o.krylov_vector(base, x, want_p=True, stats=True)
    assert ost.passes == 3
    check(y3, y_ref, tol_bar, "literal loop vs oracle")
    p3 = p3.cpu().numpy()
    assert np.abs(p3 - p_ref).max() <= tol_bar * np.abs(p_ref).max()


@pytest.mark.parametrize("prec", [0, 1])
def test_literal_loop_that_converges_reports_ok(prec):
    kv = kvmod()
    n = (12, 10, 9)
    base = np.stack(synth.base_flow(*n, synth.CC, 53))
    x = synth.krylov_input(*n, 54)[0]
    g = kv.Grid(*n, gr=1e6, precision=prec, max_passes=5)
    g.set_base_flow(torch.from_numpy(base).cuda())
    _, st = g.krylov_vector(torch.from_numpy(x).cuda(), stats=True)
    assert 1 <= st.passes < 10 and st.rel_div < 1e-12  # the paper: fewer than 10 passes


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("where", ["x", "base"])
def test_nonfinite_input_is_reported(prec, where):
    """A NaN in the input vector (or an Inf in the base velocity) must not disappear: with stats
    the call returns KV_ERR_ARG; without, it stays asynchronous and the device-side SIMPLE test
    counts the non-finite result; the grid stays usable afterwards."""
    kv = kvmod()
    n = (16, 12, 10)
    base = np.stack(synth.base_flow(*n, synth.CC, 55))
    x = synth.krylov_input(*n, 56)[0]
    bad_base, bad_x = base.copy(), x.copy()
    if where == "x":
        bad_x[1, 5, 6, 7] = np.nan
    else:
        bad_base[0, 4, 5, 6] = np.inf  # U on an interior x-face
    g = kv.Grid(*n, gr=1e6, precision=prec)
    g.set_base_flow(torch.from_numpy(bad_base).cuda())
    g.guard(reset=True)
    xt = torch.from_numpy(bad_x).cuda()
    y = g.empty(4)
    st = kv.Stats()
    rc = g.lib.kv_krylov_vector(g.h, xt.data_ptr(), y.data_ptr(), None, ctypes.byref(st))
    assert rc == -1, rc
    assert b"non-finite" in g.lib.kv_last_error(g.h)
    g.krylov_vector(xt)  # no stats: asynchronous, recorded by the guard
    gd = g.guard(reset=True)
    assert gd["nonfinite"] == 2 and gd["checks"] == 2, gd
    # the grid stays usable: a finite base flow and input give the oracle's result
    g.set_base_flow(torch.from_numpy(base).cuda())
    y = g.krylov_vector(torch.from_numpy(x).cuda()).cpu().numpy()
    check(y, Oracle(*n, gr=1e6).krylov_vector(base, x), TOL64 if prec == 0 else TOLMIX, "after NaN")
    assert g.guard()["nonfinite"] == 0


@pytest.mark.parametrize("prec", [0, 1])
def test_nan_in_an_arnoldi_step_is_reported(prec):
    kv = kvmod()
    n = (10, 9, 8)
    base = np.stack(synth.base_flow(*n, synth.CC, 57))
    g = kv.Grid(*n, gr=1e6, precision=prec)
    g.set_base_flow(torch.from_numpy(base).cuda())
    V = torch.zeros((3, 4) + g.shape, dtype=torch.float64, device="cuda")
    V[0] = torch.from_numpy(synth.krylov_input(*n, 58)[0]).cuda()
    V[0] /= torch.linalg.vector_norm(V[0])
    V[0, 2, 3, 4, 5] = float("nan")
    hcol = (ctypes.c_double * 2)()
    rc = g.lib.kv_arnoldi_step(g.h, V.data_ptr(), 0, hcol)
    if prec == 1:
        assert rc == -1  # the double-float sweeps' range check
    else:
        assert rc == 0 and not np.isfinite(hcol[1])
    assert g.guard()["nonfinite"] == 1


def test_guard_counts_one_pass_evaluations():
    kv = kvmod()
    n = (18, 16, 14)
    base = np.stack(synth.base_flow(*n, synth.CC, 59))
    xs = synth.krylov_input(*n, 60, count=3)
    for prec in (0, 1):
        g = kv.Grid(*n, gr=1e6, precision=prec)
        g.set_base_flow(torch.from_numpy(base).cuda())
        for k in range(3):
            g.krylov_vector(torch.from_numpy(xs[k]).cuda())
        gd = g.guard(reset=True)
        assert gd["checks"] == 3 and gd["failed"] == 0 and gd["nonfinite"] == 0, gd
        assert 0 < gd["worst_rel_div"] < 1e-12, gd
        assert g.guard()["checks"] == 0


def test_field_sizes_and_the_four_pointer_base_flow():
    """kv_field_sizes returns the padded lengths; kv_set_base_flow with four separate device
    fields gives the same map as the packed form."""
    kv = kvmod()
    n = (11, 9, 7)
    base = np.stack(synth.base_flow(*n, synth.AA, 61))
    x = torch.from_numpy(synth.krylov_input(*n, 62)[0]).cuda()
    g = kv.Grid(*n, bc=synth.AA, gr=1e6)
    P = (n[0] + 2) * (n[1] + 2) * (n[2] + 2)
    assert g.field_sizes() == (P, P, P, P)
    g.set_base_flow_packed(torch.from_numpy(base).cuda())
    y_packed = g.krylov_vector(x)
    fields = [torch.from_numpy(base[q].copy()).cuda() for q in range(4)]
    g2 = kv.Grid(*n, bc=synth.AA, gr=1e6)
    g2.set_base_flow_fields(*fields)
    assert torch.equal(g2.krylov_vector(x), y_packed)
    lib = g.lib
    assert lib.kv_set_base_flow(g.h, fields[0].data_ptr(), None, fields[2].data_ptr(), fields[3].data_ptr()) == -1
    assert lib.kv_field_sizes(g.h, None, None, None, None) == -1


def test_set_tuning_rejects_bad_configurations():
    kv = kvmod()
    g = kv.Grid(8, 8, 8, precision=kv.KV_PREC_MIXED)
    for bad in [((0, 8), 1, (0, 32)), ((32, 9), 1, (0, 32)), ((512, 1), 1, (0, 32)), ((32, 8), 3, (0, 32)),
                ((32, 8), 2, (0, 0)),
                ((32, 8), 0, (48, 1)), ((32, 8), 0, (128, 2)), ((32, 8), 1, (0, 0))]:
        with pytest.raises(kv.KvError) as e:
            g.set_tuning(*bad)
        assert e.value.status == -1, bad


def test_arnoldi_counts_and_device_decision_match_forced_updates():
    """The second-update decision taken on the device: forcing the update (cgs_passes = 2) and
    deciding it agree to rounding, and the counters see every fused step."""
    kv = kvmod()
    n = (14, 12, 10)
    base = np.stack(synth.base_flow(*n, synth.CC, 63))
    x0 = synth.krylov_input(*n, 64)[0]
    Hs = []
    for cgs in (0, 2):
        g = kv.Grid(*n, gr=1e6, precision=kv.KV_PREC_MIXED, cgs_passes=cgs)
        g.set_base_flow(torch.from_numpy(base).cuda())
        g.profile_enable(True)
        k = 8
        V = torch.zeros((k + 1, 4) + g.shape, dtype=torch.float64, device="cuda")
        y = g.krylov_vector(torch.from_numpy(x0).cuda())
        V[0] = y / torch.linalg.vector_norm(y)
        H = np.zeros((k + 1, k))
        for j in range(k):
            H[: j + 2, j] = g.arnoldi_step(V, j)
        steps, second = g.arnoldi_counts()
        assert steps == k
        if cgs == 2:
            assert second == k
        Vm = V.reshape(k + 1, -1)
        G = (Vm @ Vm.T).cpu().numpy()
        assert np.abs(G - np.eye(k + 1)).max() < 1e-13
        Hs.append(H)
    assert np.abs(Hs[0] - Hs[1]).max() < 1e-11 * np.abs(Hs[1]).max()


@pytest.mark.parametrize("where", ["x", "x_wall", "base"])
def test_fixed_point_operator_nonfinite_and_zero_inputs(where):
    """The fixed-point operator (variant 2) takes the input's grid from its largest kept entry: a
    NaN there makes every result non-finite (reported as the double-float path reports it), a NaN
    at an entry P_BC discards changes nothing, a zero input gives a zero result, and a non-finite
    base state falls back to the double-float march."""
    kv = kvmod()
    n = (12, 12, 12)
    base = np.stack(synth.base_flow(*n, synth.CC, 65))
    x = synth.krylov_input(*n, 66)[0]
    g = kv.Grid(*n, gr=1e6, precision=kv.KV_PREC_MIXED)
    g.set_tuning(apply_block=(32, 8), df_variant=2, df_block=(0, 8))
    bad_base, bad_x = base.copy(), x.copy()
    if where == "x":
        bad_x[3, 5, 6, 7] = np.nan
    elif where == "x_wall":
        bad_x[0, 4, 5, 0] = np.nan  # u at the wall face i = 0: not a degree of freedom
    else:
        bad_base[2, 4, 5, 6] = np.inf
    g.set_base_flow(torch.from_numpy(bad_base).cuda())
    xt = torch.from_numpy(bad_x).cuda()
    y = g.empty(4)
    st = kv.Stats()
    rc = g.lib.kv_krylov_vector(g.h, xt.data_ptr(), y.data_ptr(), None, ctypes.byref(st))
    if where == "x_wall":
        assert rc == 0
        check(y.cpu().numpy(), Oracle(*n, gr=1e6).krylov_vector(base, bad_x), TOLMIX, "NaN at a wall face")
    else:
        assert rc == -1 and b"non-finite" in g.lib.kv_last_error(g.h)
    g.set_base_flow(torch.from_numpy(base).cuda())
    z = g.krylov_vector(torch.zeros_like(xt))
    assert torch.count_nonzero(z) == 0


@pytest.mark.parametrize("n,bc,gr,tproj", [CASES[0], CASES[3], CUBES[1], ((100, 100, 100), synth.CC, 2e6, 0)])
def test_both_contraction_tiles_match_oracle(n, bc, gr, tproj):
    """The tensor-core contractions with 256- and 128-column tiles (the autotuner's two widths),
    each pinned, against the oracle; both widths give the same result to rounding."""
    kv = kvmod()
    base, x, y_ref = reference(n, bc, gr, tproj)
    ys = []
    for tile in (256, 128):
        g = kv.Grid(*n, bc=bc, gr=gr, pr=0.71, tproj=tproj, precision=kv.KV_PREC_MIXED)
        g.set_contraction_tile(tile)
        g.set_base_flow(torch.from_numpy(base).cuda())
        assert g.tuning()["contraction_tile"] == tile
        y, st = g.krylov_vector(torch.from_numpy(x).cuda(), stats=True)
        assert st.device_error == 0
        y = y.cpu().numpy()
        check(y, y_ref, TOLMIX, ("tile", tile))
        ys.append(y)
    assert np.linalg.norm(ys[0] - ys[1]) <= 1e-11 * np.linalg.norm(ys[0])


def test_contraction_tile_rejects_bad_widths():
    kv = kvmod()
    g = kv.Grid(8, 8, 8, precision=kv.KV_PREC_MIXED)
    for bad in (0, 64, 192, 512):
        with pytest.raises(kv.KvError):
            g.set_contraction_tile(bad)
    g64 = kv.Grid(8, 8, 8, precision=kv.KV_PREC_FP64)
    assert g64.contraction_tile() == -1
    with pytest.raises(kv.KvError):
        g64.set_contraction_tile(128)
