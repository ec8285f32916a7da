"""Host logic of the library, on the CPU: kv_axis_data returns the per-axis data kv_create_grid
builds, so the eigen-decomposition of Eq (15) (closed form on the uniform grid, tridiagonal QL
on a grid stretched by Eq (22)) and the stretched operator weights are checked here without a
GPU: against the oracle's independent construction (dense Jacobi rotations, Gauss-Jordan), the
independent Kronecker assembly, and the definition A E = E Lambda up to n = 256."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1905_11601_gb300 import build as kvbuild
from paper_1905_11601_gb300 import kv
from tests.mac_assembly import control_volume, d1_1d, d2_1d, positions, stretched_faces

S = 0.12
EPS = np.finfo(float).eps


def kappa(lam):
    """|lambda|_max / |lambda_1|: an FP64 eigensolver resolves eigenvectors to about eps ||A|| over
    their gap, so the constant mode and the pseudo-inverse carry errors of order eps kappa."""
    return np.abs(lam).max() / abs(lam[1])


@pytest.fixture(scope="module", autouse=True)
def lib():
    kvbuild.build()
    return kv.load_library()


def neumann_dg(n, s):
    """D G along one axis with the wall faces excluded, from its two factors."""
    dx = np.diff(stretched_faces(n, s)) if s else np.full(n, 1.0 / n)
    c = positions(n, False, s)
    g = c[2:n + 1] - c[1:n]
    Dm, Gm = np.zeros((n, n - 1)), np.zeros((n - 1, n))
    for t in range(n - 1):
        Gm[t, t + 1], Gm[t, t] = 1.0 / g[t], -1.0 / g[t]
        Dm[t, t] += 1.0 / dx[t]
        Dm[t + 1, t] -= 1.0 / dx[t + 1]
    return Dm @ Gm


@pytest.mark.parametrize("n,s", [(2, 0.0), (7, 0.0), (64, 0.0), (2, S), (3, S), (17, S), (64, S), (256, S),
                                 (40, 0.05)])
def test_eigen_decomposition_of_eq15(n, s):
    E, Ei, lam, _ = kv.axis_data(n, s)
    A = neumann_dg(n, s)
    scale = np.abs(A).max()
    assert np.abs(A @ E - E * lam[None, :]).max() < 1e-12 * scale * max(1, n / 64)
    assert np.abs(Ei @ E - np.eye(n)).max() < 1e-13 * max(1, n / 16)
    assert lam[0] == 0.0 and np.all(lam[1:] < 0) and np.all(np.diff(lam) <= 0)
    assert np.abs(E[:, 0] / E[0, 0] - 1).max() < 8 * EPS * kappa(lam)  # the constant mode
    ref = np.sort(np.linalg.eigvals(A).real)[::-1]
    assert np.allclose(lam[1:], ref[1:], rtol=1e-11, atol=1e-12 * scale)


@pytest.mark.parametrize("n", [3, 8, 17, 33])
def test_matches_the_oracle_decomposition(n):
    """The library's QL route and the oracle's Jacobi + Gauss-Jordan route give the same
    pseudo-inverse of D G to the conditioning of the eigenproblem (the eigenvectors of
    near-degenerate pairs need not agree)."""
    E, Ei, lam, _ = kv.axis_data(n, S)
    o = Oracle(n, 3, 3, stretch=S)
    Eo, Eio, lo = o.axis_data(0, 0), o.axis_data(0, 1), o.axis_data(0, 2)
    assert np.allclose(lam, lo, rtol=1e-12, atol=1e-12 * np.abs(lo).max())

    def pinv(E, Ei, lam):
        li = np.zeros_like(lam)
        li[1:] = 1.0 / lam[1:]
        return E @ np.diag(li) @ Ei

    Pl, Po = pinv(E, Ei, lam), pinv(Eo, Eio, lo)
    assert np.abs(Pl - Po).max() < 8 * EPS * kappa(lo) * np.abs(Po).max()


def test_uniform_closed_form_matches_the_oracle():
    n = 24
    E, Ei, lam, _ = kv.axis_data(n, 0.0)
    o = Oracle(n, 3, 3)
    assert np.allclose(lam, o.axis_data(0, 2), rtol=1e-13, atol=1e-12)
    assert np.allclose(E, o.axis_data(0, 0), rtol=0, atol=1e-14)
    assert np.allclose(Ei, E.T, rtol=0, atol=0)  # orthogonal on the uniform grid


@pytest.mark.parametrize("n,s", [(6, S), (17, S), (9, 0.05), (8, 0.0)])
def test_weights_match_the_kronecker_assembly(n, s):
    _, _, _, w = kv.axis_data(n, s)
    for face, r1, r2 in ((False, 2, 5), (True, 8, 11)):
        D1, D2 = d1_1d(n, face, s).toarray(), d2_1d(n, face, s).toarray()
        rows = range(1, n) if face else range(1, n + 1)
        for t in rows:
            for q, off in enumerate((-1, 0, 1)):
                assert abs(w[r1 + q, t] - D1[t, t + off]) <= 1e-13 * np.abs(D1).max()
                assert abs(w[r2 + q, t] - D2[t, t + off]) <= 1e-13 * np.abs(D2).max()
    cv_cell, cv_face = control_volume(n, False, s), control_volume(n, True, s)
    assert np.allclose(w[0, 1:n + 1], 1.0 / cv_cell[1:n + 1], rtol=1e-14, atol=0)
    assert np.allclose(w[1, 1:n], 1.0 / cv_face[1:n], rtol=1e-14, atol=0)
    assert w[1, 0] == 0 and w[1, n] == 0 and w[0, 0] == 0 and w[0, n + 1] == 0


def test_bad_arguments_rejected():
    for n, s in ((1, 0.0), (1025, 0.0), (8, -0.1), (8, 0.2), (8, float("nan"))):
        with pytest.raises(kv.KvError):
            kv.axis_data(n, s)
