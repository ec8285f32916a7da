"""Host logic of the library's Arnoldi driver (paper_1905_11601_gb300/arnoldi.py), on the CPU:
the Ritz values and residual estimates of Section 3.1 from the Hessenberg matrix, the enclosing
ellipse and the wanted set of the Chebyshev-preconditioned iteration, and the checkpoint round
trip. Each is checked against a property that does not come from the code under test."""
import numpy as np
import pytest

from paper_1905_11601_gb300 import arnoldi

torch = pytest.importorskip("torch")


def dense_arnoldi(A, v0, k):
    """k steps of modified Gram-Schmidt Arnoldi with a dense matrix (numpy)."""
    n = A.shape[0]
    V = np.zeros((k + 1, n))
    H = np.zeros((k + 1, k))
    V[0] = v0 / np.linalg.norm(v0)
    for j in range(k):
        w = A @ V[j]
        for i in range(j + 1):
            H[i, j] = V[i] @ w
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        V[j + 1] = w / H[j + 1, j]
    return V, H


def test_ritz_residual_estimate_equals_the_true_residual():
    """|h_{k+1,k}| |y_k| / ||y|| is ||A x - theta x|| / ||x|| for x = V_k y (Arnoldi relation)."""
    rng = np.random.default_rng(3)
    n, k, nev = 40, 12, 4
    A = rng.standard_normal((n, n))
    V, H = dense_arnoldi(A, rng.standard_normal(n), k)
    theta, Y, res = arnoldi.ritz(H, nev)
    assert len(theta) == nev and np.all(np.diff(theta.real) <= 0)
    ev_all = np.linalg.eigvals(H[:k, :k])
    assert theta[0].real == pytest.approx(ev_all.real.max())
    for q in range(nev):
        x = V[:k].T @ Y[:, q]
        true = np.linalg.norm(A @ x - theta[q] * x) / np.linalg.norm(x)
        assert res[q] == pytest.approx(true, rel=1e-8, abs=1e-12)


def test_ritz_vector_is_the_basis_combination():
    rng = np.random.default_rng(4)
    V = torch.from_numpy(rng.standard_normal((6, 4, 3, 3, 3)))
    y = rng.standard_normal(5) + 1j * rng.standard_normal(5)
    xr, xi = arnoldi.ritz_vector(V, y)
    ref = np.tensordot(y, V[:5].numpy(), axes=1)
    assert np.allclose(xr.numpy(), ref.real) and np.allclose(xi.numpy(), ref.imag)


@pytest.mark.parametrize("seed", range(6))
def test_ellipse_encloses_and_touches_the_points(seed):
    rng = np.random.default_rng(seed)
    re = rng.uniform(-5, -1, 9)
    im = rng.uniform(0, 3, 9) * (seed % 2)  # real spectra for even seeds
    pts = np.concatenate([re + 1j * im, re - 1j * im])
    d, c2 = arnoldi._ellipse(pts)
    # recover the semi-axes: the ellipse grows a0, b0 by one factor, so c2 / (a0^2 - b0^2) is it
    a0 = max(0.5 * (re.max() - re.min()), 1e-8)
    b0 = max(np.abs(im).max(), 1e-8 * max(re.max() - re.min(), np.abs(im).max()))
    s = c2 / (a0 * a0 - b0 * b0)
    q = ((pts.real - d) ** 2 / (s * a0 * a0) + pts.imag ** 2 / (s * b0 * b0))
    assert d == pytest.approx(0.5 * (re.max() + re.min()))
    assert s >= 1.0 - 1e-12
    assert q.max() <= 1 + 1e-12  # every point inside
    assert q.max() >= 1 - 1e-12  # and the smallest such ellipse of that shape


def test_wanted_keeps_conjugate_pairs_together():
    theta = np.array([-1 + 2j, -1 - 2j, -3 + 0j, -4 + 0j])
    assert arnoldi._wanted(theta, 1) == 2
    assert arnoldi._wanted(theta, 2) == 2
    assert arnoldi._wanted(theta, 3) == 3
    real = np.array([-1.0 + 0j, -2.0 + 0j])
    assert arnoldi._wanted(real, 1) == 1
    assert arnoldi._wanted(real, 5) == 2


def test_checkpoint_round_trip(tmp_path):
    rng = np.random.default_rng(5)
    V = torch.from_numpy(rng.standard_normal((4, 4, 3, 3, 3)))
    H = rng.standard_normal((4, 3))
    p = tmp_path / "arnoldi.pt"
    arnoldi.save_state(str(p), V, H, 3)
    V2, H2, j = arnoldi.load_state(str(p), device="cpu")
    assert torch.equal(V2, V) and np.array_equal(H2, H) and j == 3
