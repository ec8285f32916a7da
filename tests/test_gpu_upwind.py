"""GPU parity of the optional first-order upwind advection (KV_ADV_UPWIND) against the FP64
oracle's upwind branch: every FP64 block shape and every mixed operator variant (double-float
and fixed-point) at ragged sizes, the Newton residual, the transpose, an autotuned mixed grid,
and the refusal of the base-flow gradient. Per-field max-abs bars as in the central tests:
1e-12 of max |y_ref_F| for FP64, 1e-9 for mixed precision."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1905_11601_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL64, TOLMIX = 1e-12, 1e-9
UP = 1

FP64_BLOCKS = [(32, 8), (64, 4), (128, 2), (32, 4), (16, 16), (256, 1)]
DF_VARIANTS = [(0, 32, 1), (0, 32, 2), (0, 64, 1), (0, 32, 4), (0, 64, 2), (0, 128, 1), (1, 0, 16), (1, 0, 32),
               (1, 0, 64), (2, 0, 8), (2, 0, 16), (2, 0, 32), (2, 0, 64)]
CASES = [((70, 65, 67), synth.CC, 2e6, 0), ((33, 18, 20), synth.AA, 3e6, 1), ((9, 130, 12), synth.AA, 3e6, 0),
         ((37, 37, 37), synth.CC, 3.3e6, 0), ((2, 3, 2), synth.CC, 1e6, 0)]
# the fixed-point operator (variant 2) serves cubes: ragged cubes against its tiles, and cubes
# whose every cell touches a wall
CUBES = [((33, 33, 33), synth.AA, 3e6, 1), ((20, 20, 20), synth.AA, 3e6, 0), ((2, 2, 2), synth.CC, 1e6, 0),
         ((3, 3, 3), synth.AA, 1e6, 1)]


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


def reference(n, bc, gr, tproj, seed=61):
    key = (n, bc, gr, tproj, seed)
    if key not in _REF:
        base = np.stack(synth.base_flow(*n, bc, seed))
        x = synth.krylov_input(*n, seed + 1)[0]
        y_ref = Oracle(*n, bc=bc, gr=gr, pr=0.71, tproj=tproj, adv=UP).krylov_vector(base, x)
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
def test_upwind_every_fp64_block_shape_matches_oracle(n, bc, gr, tproj):
    kv = kvmod()
    base, x, y_ref = reference(n, bc, gr, tproj)
    g = kv.Grid(*n, bc=bc, gr=gr, pr=0.71, tproj=tproj, advection=kv.KV_ADV_UPWIND)
    g.set_tuning(apply_block=FP64_BLOCKS[0])
    g.set_base_flow(torch.from_numpy(base).cuda())
    xt = torch.from_numpy(x).cuda()
    for blk in FP64_BLOCKS:
        g.set_tuning(apply_block=blk)
        check(g.krylov_vector(xt).cpu().numpy(), y_ref, TOL64, blk)
    # the central scheme on the same grid gives another result: the flag reaches the kernels
    c = kv.Grid(*n, bc=bc, gr=gr, pr=0.71, tproj=tproj)
    c.set_base_flow(torch.from_numpy(base).cuda())
    yc = c.krylov_vector(xt).cpu().numpy()
    assert np.linalg.norm(yc - y_ref) > 1e-4 * np.linalg.norm(y_ref)


@pytest.mark.parametrize("n,bc,gr,tproj", CASES + CUBES + [((128, 128, 128), synth.AA, 3e6, 0)])
def test_upwind_every_mixed_operator_variant_matches_oracle(n, bc, gr, tproj):
    kv = kvmod()
    base, x, y_ref = reference(n, bc, gr, tproj)
    g = kv.Grid(*n, bc=bc, gr=gr, pr=0.71, tproj=tproj, precision=kv.KV_PREC_MIXED, advection=kv.KV_ADV_UPWIND)
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
        y, st = g.krylov_vector(xt, stats=True)
        assert st.device_error == 0
        check(y.cpu().numpy(), y_ref, TOLMIX, (v, bx, by))


def test_upwind_autotuned_mixed_grid_matches_oracle():
    kv = kvmod()
    n, bc, gr = (48, 48, 48), synth.CC, 3.3e6
    base, x, y_ref = reference(n, bc, gr, 0)
    g = kv.Grid(*n, bc=bc, gr=gr, pr=0.71, precision=kv.KV_PREC_MIXED, advection=kv.KV_ADV_UPWIND)
    g.set_base_flow(torch.from_numpy(base).cuda())  # the autotuner runs here
    assert g.tuning()["df_variant"] in (0, 1, 2)
    check(g.krylov_vector(torch.from_numpy(x).cuda()).cpu().numpy(), y_ref, TOLMIX, "autotuned")


@pytest.mark.parametrize("n,bc", [((16, 16, 16), synth.CC), ((12, 10, 9), synth.AA)])
def test_upwind_newton_residual_matches_oracle(n, bc):
    kv = kvmod()
    base = np.stack(synth.base_flow(*n, bc, 5))
    g = kv.Grid(*n, bc=bc, gr=2e6, pr=0.71, advection=kv.KV_ADV_UPWIND)
    g.set_base_flow(torch.from_numpy(base).cuda())
    F, nrm = g.newton_residual(torch.from_numpy(base).cuda())
    F_ref, nrm_ref = Oracle(*n, bc=bc, gr=2e6, adv=UP).newton_residual(base)
    F = F.cpu().numpy()
    assert np.linalg.norm(F - F_ref) < TOL64 * np.linalg.norm(F_ref)
    assert abs(nrm - nrm_ref) < TOL64 * nrm_ref


@pytest.mark.parametrize("n,bc,gr", [((24, 24, 24), synth.CC, 2.5e6), ((17, 12, 9), synth.AA, 3e6)])
def test_upwind_adjoint_matches_oracle_transpose(n, bc, gr):
    kv = kvmod()
    base = np.stack(synth.base_flow(*n, bc, 91))
    y = synth.krylov_input(*n, 92)[0]
    g = kv.Grid(*n, bc=bc, gr=gr, pr=0.71, advection=kv.KV_ADV_UPWIND)
    g.set_base_flow(torch.from_numpy(base).cuda())
    z = g.krylov_vector_adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    z_ref = Oracle(*n, bc=bc, gr=gr, adv=UP).krylov_adjoint(base, y)
    assert np.linalg.norm(z - z_ref) < TOL64 * np.linalg.norm(z_ref)


def test_upwind_base_flow_gradient_is_refused():
    kv = kvmod()
    n = (8, 8, 8)
    base = np.stack(synth.base_flow(*n, synth.CC, 3))
    g = kv.Grid(*n, advection=kv.KV_ADV_UPWIND)
    g.set_base_flow(torch.from_numpy(base).cuda())
    x = torch.from_numpy(synth.krylov_input(*n, 4, 2)).cuda()
    with pytest.raises(kv.KvError):
        g.base_flow_gradient(x[0], x[1])


def test_upwind_arnoldi_steps_match_oracle():
    kv = kvmod()
    n, bc, gr = (20, 18, 16), synth.AA, 2e6
    base = np.stack(synth.base_flow(*n, bc, 7))
    o = Oracle(*n, bc=bc, gr=gr, adv=UP)
    g = kv.Grid(*n, bc=bc, gr=gr, pr=0.71, advection=kv.KV_ADV_UPWIND)
    g.set_base_flow(torch.from_numpy(base).cuda())
    k = 4
    v0 = o.project_input(synth.krylov_input(*n, 8)[0])
    V = np.zeros((k + 1, 4) + o.shape)
    V[0] = v0 / np.linalg.norm(v0)
    Vd = torch.from_numpy(V.copy()).cuda()
    for j in range(k):
        h = g.arnoldi_step(Vd, j)
        h_ref = o.arnoldi_step(base, V, j)  # the oracle continues from the GPU basis
        assert np.abs(h - h_ref).max() < 1e-10 * np.abs(h_ref).max(), j
        V[j + 1] = Vd[j + 1].cpu().numpy()
