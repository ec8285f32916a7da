"""The delayed classical Gram-Schmidt of kv_arnoldi_run, restated in numpy with the oracle's
Krylov map as the operator, against the oracle's own Arnoldi steps (classical Gram-Schmidt
applied twice, Section 3.1), CPU only.

In exact arithmetic the two give the same basis and Hessenberg matrix: the delayed form applies
the operator to each new vector before its second projection and normalisation and corrects the
result through the Arnoldi relation of the final columns. This pins the coefficient algebra the
GPU sweeps use (kv_dcgs.cu) independently of any GPU code; the GPU run is compared with the oracle
in tests/test_gpu_arnoldi_run.py."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1905_11601_gb300 import synth


def delayed_cgs2(A, v0, m):
    """m Arnoldi steps; A: a function of one packed vector (flattened here)."""
    n = v0.size
    V = np.zeros((m + 1, n))
    H = np.zeros((m + 1, m))
    V[0] = v0 / np.linalg.norm(v0)
    for j in range(m):
        u = V[j].copy()
        w = A(u)
        Vj = V[:j]
        first = j == 0
        a = np.zeros(j) if first else Vj @ u
        b = Vj @ w
        beta = 1.0
        if not first:
            beta = np.sqrt(u @ u - a @ a)
            H[:j, j - 1] += a          # the deferred second projection of u_j
            H[j, j - 1] = beta
        d = H[:j + 1, :j] @ a          # A v_j = (w - [V, v_j] d) / beta
        h = np.empty(j + 1)
        h[:j] = (b - d[:j]) / beta
        h[j] = ((u @ w - a @ b) / beta - d[j]) / beta
        H[:j + 1, j] = h               # provisional: completed in the next step
        kappa = d[j] / beta + h[j]
        e = d[:j] / beta + h[:j] - a * kappa / beta
        V[j] = u / beta - (a / beta) @ Vj
        V[j + 1] = w / beta - (kappa / beta) * u - e @ Vj
    u = V[m].copy()
    a = V[:m] @ u
    beta = np.sqrt(u @ u - a @ a)
    H[:m, m - 1] += a
    H[m, m - 1] = beta
    V[m] = (u - a @ V[:m]) / beta
    return V, H


@pytest.mark.parametrize("n,bc,tproj", [((6, 6, 6), synth.CC, 0), ((5, 6, 4), synth.AA, 1)])
def test_delayed_gram_schmidt_equals_the_oracles_arnoldi(n, bc, tproj):
    o = Oracle(*n, bc=bc, gr=1e6, tproj=tproj)
    base = np.stack(synth.base_flow(*n, bc, 51))
    shape = (4,) + o.shape
    v0 = o.project_input(synth.krylov_input(*n, 52)[0]).ravel()
    m = 8

    def A(x):
        return o.krylov_vector(base, x.reshape(shape)).ravel()

    V, H = delayed_cgs2(A, v0, m)
    Vr = np.zeros((m + 1,) + shape)
    Vr[0] = (v0 / np.linalg.norm(v0)).reshape(shape)
    Hr = np.zeros((m + 1, m))
    for j in range(m):
        Hr[: j + 2, j] = o.arnoldi_step(base, Vr, j)
    assert np.abs(H - Hr).max() < 1e-11 * np.abs(Hr).max()
    assert np.abs(V - Vr.reshape(m + 1, -1)).max() < 1e-10
    assert np.abs(V @ V.T - np.eye(m + 1)).max() < 1e-13


def test_delayed_gram_schmidt_on_a_dense_operator():
    """A nonsymmetric dense operator with a spread spectrum: basis, Hessenberg matrix and the
    Arnoldi relation against classical Gram-Schmidt applied twice (numpy)."""
    rng = np.random.default_rng(3)
    n, m = 400, 24
    M = rng.standard_normal((n, n)) / np.sqrt(n) + np.diag(np.linspace(-3.0, 1.0, n))
    v0 = rng.standard_normal(n)
    V, H = delayed_cgs2(lambda x: M @ x, v0, m)
    Vr = np.zeros((m + 1, n))
    Hr = np.zeros((m + 1, m))
    Vr[0] = v0 / np.linalg.norm(v0)
    for j in range(m):
        w = M @ Vr[j]
        h = Vr[: j + 1] @ w
        w = w - h @ Vr[: j + 1]
        c = Vr[: j + 1] @ w
        w = w - c @ Vr[: j + 1]
        Hr[: j + 1, j] = h + c
        Hr[j + 1, j] = np.linalg.norm(w)
        Vr[j + 1] = w / Hr[j + 1, j]
    assert np.abs(H - Hr).max() < 1e-12
    assert np.abs(V - Vr).max() < 1e-12
    assert np.linalg.norm(M @ V[:m].T - V.T @ H) < 1e-13 * np.linalg.norm(M @ V[:m].T)
