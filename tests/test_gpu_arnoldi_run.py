"""kv_arnoldi_run (m Arnoldi steps with the delayed classical Gram-Schmidt) on the GPU.

Against the oracle: each Hessenberg column of a run equals the oracle's Arnoldi step taken on
the run's own basis up to that column (classical Gram-Schmidt applied twice, Section 3.1; the
comparison follows the basis, so rounding does not accumulate into it). Also: orthonormality,
the Arnoldi relation through the library's Krylov map, agreement with step-by-step
kv_arnoldi_step, a run continued from an earlier one, and the argument and range errors. Both
precisions."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1905_11601_gb300 import synth

pytestmark = pytest.mark.gpu
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


def setup(n, bc, gr, prec, seed, tproj=0):
    kv = kvmod()
    base = np.stack(synth.base_flow(*n, bc, seed))
    g = kv.Grid(*n, bc=bc, gr=gr, pr=0.71, tproj=tproj,
                precision=kv.KV_PREC_MIXED if prec == "mixed" else kv.KV_PREC_FP64)
    g.set_base_flow(torch.from_numpy(base).cuda())
    o = Oracle(*n, bc=bc, gr=gr, pr=0.71, tproj=tproj)
    v0 = o.project_input(synth.krylov_input(*n, seed + 1)[0])
    return g, o, base, v0 / np.linalg.norm(v0)


@pytest.mark.parametrize("n,bc,tproj", [((16, 16, 16), synth.CC, 0), ((33, 18, 20), synth.AA, 1)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_run_columns_match_the_oracles_arnoldi_step(n, bc, tproj, prec):
    g, o, base, v0 = setup(n, bc, 2e6, prec, 71, tproj)
    m = 12
    V = torch.zeros((m + 1, 4) + o.shape, dtype=torch.float64, device="cuda")
    V[0] = torch.from_numpy(v0)
    H = g.arnoldi_run(V, 0, m)
    Vn = V.cpu().numpy()
    # the mixed Krylov map is within 1e-9 of the FP64 one (in practice about 5e-13)
    th, tv = (1e-10, 1e-8) if prec == "fp64" else (1e-9, 1e-7)
    for j in range(m):
        Vr = np.zeros((j + 2, 4) + o.shape)
        Vr[: j + 1] = Vn[: j + 1]
        h_ref = o.arnoldi_step(base, Vr, j)
        assert np.abs(H[: j + 2, j] - h_ref).max() < th * np.abs(h_ref).max(), j
        # and the new vector: the oracle's, from the run's own basis
        assert np.abs(Vr[j + 1] - Vn[j + 1]).max() < tv * np.abs(Vr[j + 1]).max(), j
    Vm = V.reshape(m + 1, -1)
    G = (Vm @ Vm.T).cpu().numpy()
    assert np.abs(G - np.eye(m + 1)).max() < 1e-13
    assert np.all(np.tril(H, -2) == 0)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-9)])
def test_run_satisfies_the_arnoldi_relation(prec, tol):
    g, o, base, v0 = setup((24, 24, 24), synth.CC, 3e6, prec, 73)
    m = 20
    V = torch.zeros((m + 1, 4) + o.shape, dtype=torch.float64, device="cuda")
    V[0] = torch.from_numpy(v0)
    H = g.arnoldi_run(V, 0, m)
    AV = torch.stack([g.krylov_vector(V[j]) for j in range(m)]).reshape(m, -1)
    R = AV - (torch.from_numpy(H.T.copy()).cuda() @ V.reshape(m + 1, -1))
    assert (torch.linalg.norm(R) / torch.linalg.norm(AV)).item() < tol
    Vm = V.reshape(m + 1, -1)
    orth = (Vm @ Vm.T - torch.eye(m + 1, dtype=torch.float64, device="cuda")).abs().max().item()
    assert orth < 1e-13


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_run_agrees_with_stepwise_arnoldi(prec):
    g, o, base, v0 = setup((20, 20, 20), synth.AA, 2e6, prec, 75)
    m = 10
    V1 = torch.zeros((m + 1, 4) + o.shape, dtype=torch.float64, device="cuda")
    V1[0] = torch.from_numpy(v0)
    V2 = V1.clone()
    H1 = g.arnoldi_run(V1, 0, m)
    H2 = np.zeros((m + 1, m))
    for j in range(m):
        H2[: j + 2, j] = g.arnoldi_step(V2, j)
    assert np.abs(H1 - H2).max() < 1e-10 * np.abs(H2).max()
    assert (V1 - V2).abs().max().item() < 1e-8


def test_run_continues_an_earlier_run():
    g, o, base, v0 = setup((16, 16, 16), synth.CC, 1e6, "mixed", 77)
    m = 12
    V1 = torch.zeros((m + 1, 4) + o.shape, dtype=torch.float64, device="cuda")
    V1[0] = torch.from_numpy(v0)
    V2 = V1.clone()
    H1 = g.arnoldi_run(V1, 0, m)
    Ha = g.arnoldi_run(V2, 0, 5)
    H2 = g.arnoldi_run(V2, 5, m - 5, Ha)
    assert np.abs(H1 - H2).max() < 1e-10 * np.abs(H1).max()
    assert (V1 - V2).abs().max().item() < 1e-8


@pytest.mark.parametrize("prec,th", [("fp64", 1e-10), ("mixed", 1e-9)])
def test_run_beyond_one_chunk(prec, th):
    """40 steps: the sweeps run in chunks of 24 basis vectors from step 25 on."""
    g, o, base, v0 = setup((12, 12, 12), synth.AA, 2e6, prec, 81)
    m = 40
    V = torch.zeros((m + 1, 4) + o.shape, dtype=torch.float64, device="cuda")
    V[0] = torch.from_numpy(v0)
    H = g.arnoldi_run(V, 0, m)
    Vn = V.cpu().numpy()
    for j in (0, 1, 23, 24, 25, 30, 39):
        Vr = np.zeros((j + 2, 4) + o.shape)
        Vr[: j + 1] = Vn[: j + 1]
        h_ref = o.arnoldi_step(base, Vr, j)
        assert np.abs(H[: j + 2, j] - h_ref).max() < th * np.abs(h_ref).max(), j
    Vm = V.reshape(m + 1, -1)
    orth = (Vm @ Vm.T - torch.eye(m + 1, dtype=torch.float64, device="cuda")).abs().max().item()
    assert orth < 1e-13
    AV = torch.stack([g.krylov_vector(V[j]) for j in range(m)]).reshape(m, -1)
    R = AV - (torch.from_numpy(H.T.copy()).cuda() @ Vm)
    assert (torch.linalg.norm(R) / torch.linalg.norm(AV)).item() < (1e-12 if prec == "fp64" else 1e-9)


def test_run_errors():
    kv = kvmod()
    g, o, base, v0 = setup((8, 8, 8), synth.CC, 1e6, "mixed", 79)
    V = torch.zeros((26, 4) + o.shape, dtype=torch.float64, device="cuda")
    V[0] = torch.from_numpy(v0)
    with pytest.raises(kv.KvError):
        g.arnoldi_run(V, 0, 0)
    V[0].view(-1)[123] = float("nan")  # a non-finite start vector: reported, no hang
    with pytest.raises(kv.KvError):
        g.arnoldi_run(V, 0, 3)
