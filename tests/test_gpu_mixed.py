"""GPU parity of the mixed-precision path (tensor-core TPF contractions in BF16 slices with
FP32 accumulation, refined with an FP64 residual) against the FP64 oracle.

Tolerance: relative 2-norm error <= 1e-9 (the mixed-form bar)."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1905_11601_gb300 import synth

pytestmark = pytest.mark.gpu
RTOL_MIXED = 1e-9
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_11601_gb300 import build
    build.build()


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


def grid(n, bc, gr, tproj=0, sweeps=0):
    from paper_1905_11601_gb300 import kv
    return kv.Grid(*n, bc=bc, gr=gr, pr=0.71, tproj=tproj, precision=kv.KV_PREC_MIXED, refine_sweeps=sweeps)


@pytest.mark.parametrize("n,bc,gr,tproj", [((16, 16, 16), synth.CC, 1e6, 0), ((33, 18, 20), synth.AA, 3e6, 0),
                                           ((70, 65, 67), synth.CC, 2e6, 0), ((9, 130, 12), synth.AA, 3e6, 1),
                                           ((2, 3, 2), synth.CC, 1e6, 0)])
def test_mixed_krylov_vector_matches_oracle(n, bc, gr, tproj):
    base = np.stack(synth.base_flow(*n, bc, 17))
    x = synth.krylov_input(*n, 18)[0]
    g = grid(n, bc, gr, tproj)
    g.set_base_flow(torch.from_numpy(base).cuda())
    y, st = g.krylov_vector(torch.from_numpy(x).cuda(), stats=True)
    assert st.device_error == 0
    y_ref = Oracle(*n, bc=bc, gr=gr, pr=0.71, tproj=tproj).krylov_vector(base, x)
    err = rel(y.cpu().numpy(), y_ref)
    assert err < RTOL_MIXED, err
    ok = field_max_ok(y.cpu().numpy(), y_ref, RTOL_MIXED)
    assert ok[0], ok


def test_mixed_at_128_insulated_matches_oracle():
    w = synth.WORKLOADS["cube128_aa"]
    n = (w.nx, w.ny, w.nz)
    base, x = synth.workload_arrays(w)
    base = np.stack(base)
    g = grid(n, w.bc, w.gr)
    g.set_base_flow(torch.from_numpy(base).cuda())
    y, st = g.krylov_vector(torch.from_numpy(x[0]).cuda(), stats=True)
    assert st.device_error == 0
    y_ref = Oracle(*n, bc=w.bc, gr=w.gr, pr=w.pr).krylov_vector(base, x[0])
    assert rel(y.cpu().numpy(), y_ref) < RTOL_MIXED
    ok = field_max_ok(y.cpu().numpy(), y_ref, RTOL_MIXED)
    assert ok[0], ok


def test_mixed_at_256_matches_fp64_path():
    """At the benchmark size the FP64 GPU path (itself checked against the oracle) is the
    reference; the error is reported per result."""
    from paper_1905_11601_gb300 import kv
    w = synth.WORKLOADS["cube256_cc"]
    n = (w.nx, w.ny, w.nz)
    base, x = synth.workload_arrays(w)
    bt = torch.from_numpy(np.stack(base)).cuda()
    xt = torch.from_numpy(x[0]).cuda()
    g64 = kv.Grid(*n, bc=w.bc, gr=w.gr, pr=w.pr)
    g64.set_base_flow(bt)
    y64 = g64.krylov_vector(xt)
    del g64
    gm = grid(n, w.bc, w.gr)
    gm.set_base_flow(bt)
    ym, st = gm.krylov_vector(xt, stats=True)
    assert st.device_error == 0
    err = (torch.linalg.vector_norm(ym - y64) / torch.linalg.vector_norm(y64)).item()
    assert err < RTOL_MIXED, err


def test_mixed_arnoldi_step_orthonormal():
    n = (24, 24, 24)
    base = np.stack(synth.base_flow(*n, synth.CC, 3))
    g = grid(n, synth.CC, 1e6)
    g.set_base_flow(torch.from_numpy(base).cuda())
    k = 6
    V = torch.zeros((k + 1, 4) + g.shape, dtype=torch.float64, device="cuda")
    y = g.krylov_vector(torch.from_numpy(synth.krylov_input(*n, 4)[0]).cuda())
    V[0] = y / torch.linalg.vector_norm(y)
    for j in range(k):
        g.arnoldi_step(V, j)
    Vm = V.reshape(k + 1, -1)
    assert (Vm @ Vm.T - torch.eye(k + 1, dtype=torch.float64, device="cuda")).abs().max().item() < 1e-12


def _cgs2_fp64(Vj, w):
    """Two-pass classical Gram-Schmidt of w against the orthonormal rows of Vj, in FP64 numpy:
    the coefficients V^T w (both passes summed), the remaining norm and the new unit vector."""
    h1 = Vj @ w
    w1 = w - Vj.T @ h1
    h2 = Vj @ w1
    w2 = w1 - Vj.T @ h2
    beta = np.linalg.norm(w2)
    return h1 + h2, beta, w2 / beta


def test_mixed_gram_schmidt_matches_fp64_definition():
    """The double-float Gram-Schmidt sweeps of the mixed-precision Arnoldi step against the
    FP64 definition applied to the same w = A V_j (the operator is deterministic, so the vector
    the step orthogonalises is recomputed exactly). Covers every basis size of the fused
    kernels (1..24) and several vector entries per thread."""
    n = (70, 65, 67)
    base = np.stack(synth.base_flow(*n, synth.CC, 21))
    g = grid(n, synth.CC, 2e6)
    g.set_base_flow(torch.from_numpy(base).cuda())
    k = 24
    V = torch.zeros((k + 1, 4) + g.shape, dtype=torch.float64, device="cuda")
    y = g.krylov_vector(torch.from_numpy(synth.krylov_input(*n, 22)[0]).cuda())
    V[0] = y / torch.linalg.vector_norm(y)
    for j in range(k):
        w = g.krylov_vector(V[j].contiguous()).reshape(-1).cpu().numpy()
        Vj = V[: j + 1].reshape(j + 1, -1).cpu().numpy()
        h_ref, beta_ref, q_ref = _cgs2_fp64(Vj, w)
        h = g.arnoldi_step(V, j)
        nw = np.linalg.norm(w)
        # each double-float term carries < 2^-46 relative error: |dh| <= 2^-46 ||w|| by Cauchy-Schwarz
        assert np.abs(h[: j + 1] - h_ref).max() < 2e-13 * nw, j
        assert abs(h[j + 1] - beta_ref) < 2e-13 * nw, j
        q = V[j + 1].reshape(-1).cpu().numpy()
        assert np.linalg.norm(q - q_ref) < 1e-12 * nw / beta_ref, j


def test_mixed_gram_schmidt_range_error():
    """A new vector with entries beyond the double-float sweeps' range is reported, not
    silently orthogonalised; the grid stays usable."""
    from paper_1905_11601_gb300 import kv
    n = (16, 16, 16)
    base = np.stack(synth.base_flow(*n, synth.CC, 23))
    g = grid(n, synth.CC, 1e6)
    g.set_base_flow(torch.from_numpy(base).cuda())
    V = torch.zeros((2, 4) + g.shape, dtype=torch.float64, device="cuda")
    y = g.krylov_vector(torch.from_numpy(synth.krylov_input(*n, 24)[0]).cuda())
    V[0] = y / torch.linalg.vector_norm(y) * 2.0 ** 60
    with pytest.raises(kv.KvError, match="range"):
        g.arnoldi_step(V, 0)
    V[0] = y / torch.linalg.vector_norm(y)
    h = g.arnoldi_step(V, 0)
    assert np.isfinite(h).all() and h[1] > 0


def test_refinement_sweeps_converge():
    """One tensor-core sweep (FP64 store of phi), two (FP32 phi, then phi32 + D) and three (a
    further FP64 accumulation, residual read from FP64 phi): each refinement sweep shrinks the
    error by about the accuracy of one BF16-slice solve, and two already meet the bar."""
    n = (40, 36, 44)
    base = np.stack(synth.base_flow(*n, synth.CC, 31))
    x = synth.krylov_input(*n, 32)[0]
    y_ref = Oracle(*n, gr=2e6, pr=0.71).krylov_vector(base, x)
    errs = []
    for sweeps in (1, 2, 3):
        g = grid(n, synth.CC, 2e6, sweeps=sweeps)
        g.set_base_flow(torch.from_numpy(base).cuda())
        y, st = g.krylov_vector(torch.from_numpy(x).cuda(), stats=True)
        assert st.device_error == 0
        errs.append(rel(y.cpu().numpy(), y_ref))
    assert errs[0] < 1e-3, errs
    assert errs[1] < RTOL_MIXED and errs[2] < RTOL_MIXED, errs
    assert errs[1] < 1e-3 * errs[0], errs


@pytest.mark.parametrize("prec", [0, 1])
def test_second_update_criterion_matches_forced_reorthogonalisation(prec):
    """The second Gram-Schmidt update is applied only when the measured second-pass coefficients
    exceed the sweeps' rounding level; the basis and Hessenberg matrix then agree to rounding
    with the ones built when it is always applied (cgs_passes = 2)."""
    from paper_1905_11601_gb300 import kv
    n = (36, 30, 34)
    base = np.stack(synth.base_flow(*n, synth.CC, 41))
    x = synth.krylov_input(*n, 42)[0]
    k = 16
    out = []
    for cgs in (0, 2):
        g = kv.Grid(*n, gr=2e6, pr=0.71, precision=prec, cgs_passes=cgs)
        g.set_base_flow(torch.from_numpy(base).cuda())
        V = torch.zeros((k + 1, 4) + g.shape, dtype=torch.float64, device="cuda")
        y = g.krylov_vector(torch.from_numpy(x).cuda())
        V[0] = y / torch.linalg.vector_norm(y)
        H = np.zeros((k + 1, k))
        for j in range(k):
            H[: j + 2, j] = g.arnoldi_step(V, j)
        out.append((H, V.reshape(k + 1, -1).cpu().numpy()))
    (H0, V0), (H2, V2) = out
    assert np.abs(H0 - H2).max() < 1e-12 * np.abs(H2).max()
    assert np.abs(V0 - V2).max() < 1e-10
    G = V0 @ V0.T
    assert np.abs(G - np.eye(k + 1)).max() < 1e-13


@pytest.mark.parametrize("prec", [0, 1])
def test_gram_schmidt_beyond_24_matches_fp64_definition(prec):
    """Basis sizes beyond the fused kernels (25..52: inner products in chunks of 24 vectors, the
    update as a sweep of its own, on both pipes in mixed precision) against the FP64 definition
    applied to the same w = A V_j, as above; then the orthogonality of the whole basis."""
    from paper_1905_11601_gb300 import kv
    n = (20, 18, 16)
    base = np.stack(synth.base_flow(*n, synth.CC, 25))
    g = kv.Grid(*n, gr=2e6, pr=0.71, precision=prec)
    g.set_base_flow(torch.from_numpy(base).cuda())
    k = 52
    V = torch.zeros((k + 1, 4) + g.shape, dtype=torch.float64, device="cuda")
    y = g.krylov_vector(torch.from_numpy(synth.krylov_input(*n, 26)[0]).cuda())
    V[0] = y / torch.linalg.vector_norm(y)
    bar = 2e-13 if prec == 1 else 1e-14
    for j in range(k):
        if j < 24:
            g.arnoldi_step(V, j)
            continue
        w = g.krylov_vector(V[j].contiguous()).reshape(-1).cpu().numpy()
        Vj = V[: j + 1].reshape(j + 1, -1).cpu().numpy()
        h_ref, beta_ref, q_ref = _cgs2_fp64(Vj, w)
        h = g.arnoldi_step(V, j)
        nw = np.linalg.norm(w)
        assert np.abs(h[: j + 1] - h_ref).max() < bar * nw, j
        assert abs(h[j + 1] - beta_ref) < bar * nw, j
        q = V[j + 1].reshape(-1).cpu().numpy()
        assert np.linalg.norm(q - q_ref) < 50 * bar * nw / beta_ref, j
    Vm = V.reshape(k + 1, -1)
    G = (Vm @ Vm.T).cpu().numpy()
    assert np.abs(G - np.eye(k + 1)).max() < 1e-13
