"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerance: relative 2-norm error <= 1e-12 for the FP64 path (the oracle and the kernels sum
in different orders; the Neumann Poisson solve amplifies rounding in its lowest modes)."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1905_11601_gb300 import synth

pytestmark = pytest.mark.gpu
RTOL = 1e-12

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_11601_gb300 import build
    build.build()


def kvmod():
    from paper_1905_11601_gb300 import kv
    return kv


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def field_max_ok(y, y_ref, tol):
    """Per field F: max |y_F - y_ref_F| <= tol * max |y_ref_F| (catches errors confined to a wall
    or a tile's tail, which a 2-norm over the whole vector can hide)."""
    for F in range(4):
        m = np.abs(y_ref[F]).max()
        e = np.abs(y[F] - y_ref[F]).max()
        if e > tol * m:
            return False, F, e / m if m else e
    return True, None, 0.0


def setup(n, bc, gr, seed, tproj=0, count=1):
    base = np.stack(synth.base_flow(*n, bc, seed))
    x = synth.krylov_input(*n, seed, count)
    g = kvmod().Grid(*n, bc=bc, gr=gr, pr=0.71, tproj=tproj)
    g.set_base_flow(torch.from_numpy(base).cuda())
    return g, base, x


CASES = [((16, 16, 16), synth.CC, 1e6, 0), ((5, 4, 6), synth.CC, 2e6, 0), ((70, 65, 67), synth.CC, 2e6, 0),
         ((33, 18, 20), synth.AA, 3e6, 0), ((33, 18, 20), synth.AA, 3e6, 1), ((2, 3, 2), synth.AA, 1e6, 0)]


@pytest.mark.parametrize("n,bc,gr,tproj", CASES)
def test_krylov_vector_matches_oracle(n, bc, gr, tproj):
    g, base, x = setup(n, bc, gr, 11601, tproj)
    y, st = g.krylov_vector(torch.from_numpy(x[0]).cuda(), p=g.empty(), stats=True)
    o = Oracle(*n, bc=bc, gr=gr, pr=0.71, tproj=tproj)
    y_ref, p_ref = o.krylov_vector(base, x[0], want_p=True)
    y_gpu = y.cpu().numpy()
    assert rel(y_gpu, y_ref) < RTOL
    for F in range(4):
        assert rel(y_gpu[F], y_ref[F]) < 10 * RTOL or np.linalg.norm(y_ref[F]) == 0
    ok = field_max_ok(y_gpu, y_ref, RTOL)
    assert ok[0], ok
    assert st.passes == 1 and st.rel_div < 1e-13


@pytest.mark.parametrize("n,bc", [((16, 16, 16), synth.CC), ((20, 9, 14), synth.AA)])
def test_pressure_matches_oracle(n, bc):
    g, base, x = setup(n, bc, 1e6, 7)
    p = g.empty()
    g.krylov_vector(torch.from_numpy(x[0]).cuda(), p=p)
    _, p_ref = Oracle(*n, bc=bc, gr=1e6).krylov_vector(base, x[0], want_p=True)
    assert np.abs(p.cpu().numpy() - p_ref).max() < 1e-12 * np.abs(p_ref).max()


def test_y_independent_of_output_contents_and_repeatable():
    n = (24, 20, 18)
    g, base, x = setup(n, synth.CC, 1e6, 3)
    xt = torch.from_numpy(x[0]).cuda()
    y1 = g.krylov_vector(xt)
    y2 = torch.full_like(y1, float("nan"))
    g.krylov_vector(xt, y=y2)
    assert torch.equal(y1, y2)


@pytest.mark.parametrize("n,bc", [((16, 16, 16), synth.CC), ((12, 10, 9), synth.AA)])
def test_newton_residual_matches_oracle(n, bc):
    g, base, _ = setup(n, bc, 2e6, 5)
    F, nrm = g.newton_residual(torch.from_numpy(base).cuda())
    F_ref, nrm_ref = Oracle(*n, bc=bc, gr=2e6).newton_residual(base)
    assert rel(F.cpu().numpy(), F_ref) < RTOL
    assert abs(nrm - nrm_ref) < RTOL * nrm_ref


def test_arnoldi_steps_match_oracle():
    n = (16, 16, 16)
    g, base, x = setup(n, synth.CC, 1e6, 11601)
    o = Oracle(*n, gr=1e6)
    k = 20
    v0 = o.project_input(x[0])
    v0 /= np.linalg.norm(v0)
    V_ref = np.zeros((k + 1, 4) + o.shape)
    V_ref[0] = v0
    V = torch.zeros((k + 1, 4) + o.shape, dtype=torch.float64, device="cuda")
    V[0] = torch.from_numpy(v0)
    for j in range(k):
        h_gpu = g.arnoldi_step(V, j)
        h_ref = o.arnoldi_step(base, V_ref, j)
        # the basis drifts by rounding as j grows; compare each step against the oracle fed the
        # same V (copy the GPU basis into the oracle's)
        assert np.abs(h_gpu - h_ref).max() < 1e-10 * np.abs(h_ref).max(), j
        V_ref[j + 1] = V[j + 1].cpu().numpy()
    Vm = V.reshape(k + 1, -1)
    G = (Vm @ Vm.T).cpu().numpy()
    assert np.abs(G - np.eye(k + 1)).max() < 1e-12


@pytest.mark.parametrize("prec,cgs", [(0, 0), (1, 0), (1, 2)])
def test_arnoldi_orthogonality_over_a_long_basis(prec, cgs):
    """Both Gram-Schmidt code paths (fused for <= 24 vectors, unfused beyond) keep the basis
    orthonormal to rounding."""
    from paper_1905_11601_gb300 import kv
    n = (20, 18, 16)
    base = np.stack(synth.base_flow(*n, synth.CC, 61))
    g = kv.Grid(*n, gr=1e6, precision=prec, cgs_passes=cgs)
    g.set_base_flow(torch.from_numpy(base).cuda())
    k = 30
    V = torch.zeros((k + 1, 4) + g.shape, dtype=torch.float64, device="cuda")
    y = g.krylov_vector(torch.from_numpy(synth.krylov_input(*n, 62)[0]).cuda())
    V[0] = y / torch.linalg.vector_norm(y)
    H = np.zeros((k + 1, k))
    for j in range(k):
        H[: j + 2, j] = g.arnoldi_step(V, j)
    Vm = V.reshape(k + 1, -1)
    G = (Vm @ Vm.T).cpu().numpy()
    assert np.abs(G - np.eye(k + 1)).max() < 1e-12
    # Arnoldi relation A V_k = V_{k+1} H
    AV = torch.stack([g.krylov_vector(V[j].contiguous()) for j in range(k)]).reshape(k, -1)
    R = AV.T - Vm.T @ torch.from_numpy(H).cuda()
    assert (torch.linalg.matrix_norm(R) / torch.linalg.matrix_norm(AV)).item() < 1e-12


def test_host_buffer_entry_point_matches_device_path():
    n = (18, 16, 14)
    g, base, x = setup(n, synth.CC, 1e6, 9)
    y_dev = g.krylov_vector(torch.from_numpy(x[0]).cuda()).cpu().numpy()
    xh = torch.from_numpy(x[0].copy()).pin_memory()
    yh = torch.zeros_like(xh).pin_memory()
    g.krylov_vector_host(xh, yh)
    assert np.array_equal(yh.numpy(), y_dev)


def test_errors_are_reported():
    kv = kvmod()
    n = (8, 8, 8)
    g = kv.Grid(*n)
    x = g.empty(4)
    with pytest.raises(kv.KvError) as e:
        g.krylov_vector(x)  # no base flow yet
    assert e.value.status == -4
    g.set_base_flow(g.empty(4))
    # overlapping input and output are refused on the host
    assert g.lib.kv_krylov_vector(g.h, x.data_ptr(), x.data_ptr(), None, None) == -1
    assert b"overlap" in g.lib.kv_last_error(g.h)


@pytest.mark.parametrize("wl", ["cube100_cc", "cube256_cc"])
def test_full_size_properties(wl):
    """At the benchmark sizes: the temperature part equals the oracle's projected J x, the
    velocity is divergence-free, and v* - y_v equals the gradient of the returned pressure,
    which together fix y_v uniquely (discrete Helmholtz decomposition)."""
    w = synth.WORKLOADS[wl]
    n = (w.nx, w.ny, w.nz)
    g, base, x = setup(n, w.bc, w.gr, w.seed)
    p = g.empty()
    y = g.krylov_vector(torch.from_numpy(x[0]).cuda(), p=p).cpu().numpy()
    p = p.cpu().numpy()
    o = Oracle(*n, bc=w.bc, gr=w.gr, pr=w.pr)
    xp = o.project_input(x[0])
    ys = o.jx_raw(base, xp)
    T_ref = o.tproj_closed(ys[3])
    assert rel(y[3], T_ref) < RTOL
    nx, ny, nz = n
    u, v, ww = y[:3]
    div = ((u[1:-1, 1:-1, 1:-1] - u[1:-1, 1:-1, :-2]) * nx + (v[1:-1, 1:-1, 1:-1] - v[1:-1, :-2, 1:-1]) * ny
           + (ww[1:-1, 1:-1, 1:-1] - ww[:-2, 1:-1, 1:-1]) * nz)
    assert np.abs(div).max() / (np.abs(y[:3]).max() * max(n)) < 1e-13
    gp = np.zeros_like(y[:3])
    gp[0][1:-1, 1:-1, 1:-2] = (p[1:-1, 1:-1, 2:-1] - p[1:-1, 1:-1, 1:-2]) * nx
    gp[1][1:-1, 1:-2, 1:-1] = (p[1:-1, 2:-1, 1:-1] - p[1:-1, 1:-2, 1:-1]) * ny
    gp[2][1:-2, 1:-1, 1:-1] = (p[2:-1, 1:-1, 1:-1] - p[1:-2, 1:-1, 1:-1]) * nz
    assert rel(ys[:3] - y[:3], gp) < 1e-11
