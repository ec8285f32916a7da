"""Eigenvalue problem Eq (10) through the GPU map: 60 Arnoldi steps on the 100^3 grid
(Gr = 2e6, CC), the 6 rightmost Ritz values, and the residual the paper monitors
(||A X - theta X|| / ||X||), computed explicitly with the Krylov map and compared with the
Arnoldi relation's estimate. The FP64 and mixed-precision paths give the same Ritz values."""
import numpy as np
import pytest

from paper_1905_11601_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_11601_gb300 import build
    build.build()


def run(precision, k=60, nev=6):
    from paper_1905_11601_gb300 import kv
    from paper_1905_11601_gb300.arnoldi import arnoldi, ritz, ritz_vector
    w = synth.WORKLOADS["cube100_cc"]
    base, x = synth.workload_arrays(w)
    g = kv.Grid(w.nx, w.ny, w.nz, bc=w.bc, gr=w.gr, pr=w.pr, precision=precision)
    g.set_base_flow(torch.from_numpy(np.stack(base)).cuda())
    v0 = g.krylov_vector(torch.from_numpy(x[0]).cuda())
    V, H = arnoldi(g, v0, k)
    theta, Y, res = ritz(H, nev)
    # explicit residual of the leading Ritz pair: || A X - theta X || / || X ||
    xr, xi = ritz_vector(V, Y[:, 0])
    axr, axi = g.krylov_vector(xr.contiguous()), g.krylov_vector(xi.contiguous())
    t = theta[0]
    rr = axr - (t.real * xr - t.imag * xi)
    ri = axi - (t.real * xi + t.imag * xr)
    expl = torch.sqrt((rr ** 2).sum() + (ri ** 2).sum()) / torch.sqrt((xr ** 2).sum() + (xi ** 2).sum())
    return theta, res, expl.item(), V


def test_rightmost_ritz_values_and_residuals():
    th64, res64, expl64, V = run(0)
    Vm = V.reshape(V.shape[0], -1)
    G = (Vm @ Vm.T).cpu().numpy()
    assert np.abs(G - np.eye(G.shape[0])).max() < 1e-11
    # the Arnoldi estimate of the residual matches the explicit residual of the Ritz pair
    assert abs(expl64 - res64[0]) < 1e-8 * max(abs(th64[0]), 1.0)
    del V
    thm, resm, explm, V = run(1)
    del V
    assert np.allclose(thm, th64, rtol=1e-7, atol=1e-9)
    assert abs(explm - resm[0]) < 1e-8 * max(abs(thm[0]), 1.0)
