"""Pins of the oracle's Krylov solvers and Newton iteration (oracle/solvers.py) against facts fixed
by linear algebra: a direct dense solve, the least-squares characterisation of a GMRES cycle,
the finite termination of BiCG for a matrix with two distinct eigenvalues, manufactured
solutions on the Krylov-vector map, and the quadratic convergence of Newton's method (Section 2,
steps 1-4). CPU only."""
import importlib.util
import os

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1905_11601_gb300 import synth

# the solvers under test: oracle/solvers.py, or a copy with a planted mistake
# (tests/test_oracle_solver_mutations.py sets KV_SOLVERS_PATH)
_path = os.environ.get("KV_SOLVERS_PATH")
if _path:
    _spec = importlib.util.spec_from_file_location("kv_solvers_under_test", _path)
    _solvers = importlib.util.module_from_spec(_spec)
    _spec.loader.exec_module(_solvers)
else:
    from oracle import solvers as _solvers
bicgstab2, gmres, newton = _solvers.bicgstab2, _solvers.gmres, _solvers.newton


def dense_system(n, seed):
    rng = np.random.default_rng(seed)
    A = 4.0 * np.eye(n) + rng.standard_normal((n, n)) * 0.5 / np.sqrt(n) \
        + np.triu(rng.standard_normal((n, n)), 1) * 0.3 / np.sqrt(n)
    return A, rng.standard_normal(n)


def test_gmres_dense_matches_direct_solve():
    A, b = dense_system(60, 1)
    xt = np.linalg.solve(A, b)
    x, info = gmres(lambda v: A @ v, b, np.zeros(60), m=10, max_restarts=50, tol=1e-12)
    assert info["converged"] and info["restarts"] >= 2  # restarted, not one full cycle
    assert np.linalg.norm(x - xt) < 1e-10 * np.linalg.norm(xt)
    assert np.linalg.norm(b - A @ x) <= 1e-12 * np.linalg.norm(b) * 1.01


def test_gmres_cycle_is_least_squares_minimiser_over_krylov_space():
    """One cycle of GMRES(k) from x0 = 0 returns argmin ||b - A x|| over span{b, Ab, ..,
    A^(k-1) b}; the minimiser is recomputed here from a QR-orthonormalised power basis and
    numpy's least squares, independently of the Arnoldi/Givens path."""
    A, b = dense_system(40, 2)
    k = 7
    x, info = gmres(lambda v: A @ v, b, np.zeros(40), m=k, max_restarts=1, tol=0.0)
    assert info["iterations"] == k and info["restarts"] == 1
    K = np.stack([np.linalg.matrix_power(A, i) @ b for i in range(k)], axis=1)
    Q, _ = np.linalg.qr(K)
    y, *_ = np.linalg.lstsq(A @ Q, b, rcond=None)
    assert np.linalg.norm(x - Q @ y) < 1e-10 * np.linalg.norm(x)


def test_gmres_saturation_stops_restarts():
    """A cycle that cannot reduce the residual (m = 1 on a rotation) is reported as saturated."""
    A = np.array([[0.0, 1.0], [-1.0, 0.0]])
    b = np.array([1.0, 0.0])
    x, info = gmres(lambda v: A @ v, b, np.zeros(2), m=1, max_restarts=10, tol=1e-12, sat=0.99)
    assert info["saturated"] and not info["converged"] and info["restarts"] == 1


def test_bicgstab2_dense_matches_direct_solve():
    A, b = dense_system(60, 3)
    xt = np.linalg.solve(A, b)
    x, info = bicgstab2(lambda v: A @ v, b, np.zeros(60), max_iter=200, tol=1e-12)
    assert info["converged"] and not info["breakdown"]
    assert info["matvecs"] == 4 * info["iterations"] + 2
    assert np.linalg.norm(x - xt) < 1e-10 * np.linalg.norm(xt)


def test_bicgstab2_terminates_for_two_distinct_eigenvalues():
    """A = Q diag(2, .., 2, 5, .., 5) Q^T has a degree-2 minimal polynomial, so the two BiCG steps
    of the first BiCGstab(2) iteration already give the exact solution."""
    rng = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    A = Q @ np.diag([2.0] * 13 + [5.0] * 17) @ Q.T
    b = rng.standard_normal(30)
    x, info = bicgstab2(lambda v: A @ v, b, np.zeros(30), max_iter=1, tol=0.0)
    assert info["iterations"] == 1
    assert np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-12 * np.linalg.norm(x)


def _operator_case(gr=1e4):
    n = (6, 6, 6)
    o = Oracle(*n, gr=gr)
    S = np.stack(synth.base_flow(*n, synth.CC, 41))
    z = o.project_input(synth.krylov_input(*n, 7)[0])
    x_true = o.krylov_vector(S, z)           # inside the space the Krylov vectors span
    b = o.krylov_vector(S, x_true)
    return o, S, x_true, b


def test_gmres_recovers_manufactured_solution_of_krylov_map():
    o, S, x_true, b = _operator_case()
    x, info = gmres(lambda v: o.krylov_vector(S, v), b, np.zeros_like(b), m=30, max_restarts=20, tol=1e-12)
    assert info["converged"]
    assert np.linalg.norm(x - x_true) < 1e-9 * np.linalg.norm(x_true)


def test_bicgstab2_recovers_manufactured_solution_of_krylov_map():
    o, S, x_true, b = _operator_case()
    x, info = bicgstab2(lambda v: o.krylov_vector(S, v), b, np.zeros_like(b), max_iter=200, tol=1e-12)
    assert info["converged"]
    assert np.linalg.norm(x - x_true) < 1e-9 * np.linalg.norm(x_true)


@pytest.mark.parametrize("bc", [synth.CC, synth.AA])
def test_newton_converges_quadratically_to_a_steady_state(bc):
    """Steps 1-4 of Section 2 from the synthetic base flow at Gr = 1e4: the residual falls to
    rounding, each of the last steps roughly squares it, and the returned state's residual,
    recomputed, is at rounding level."""
    n = (6, 6, 6)
    o = Oracle(*n, bc=bc, gr=1e4)
    S0 = np.stack(synth.base_flow(*n, bc, 41))
    S, info = newton(o, S0, max_newton=10, tol=1e-10, m=30, max_restarts=20, lin_tol=1e-11, sat=0.99,
                     bicg_max_iter=300)
    r = info["res_norms"]
    assert info["converged"] and 4 <= info["iterations"] <= 8
    # quadratic phase: ||F_{k+1}|| <= C ||F_k||^2 with a modest C once ||F_k|| < 1e-2
    tail = [(a, c) for a, c in zip(r[:-1], r[1:]) if a < 1e-2 and c > 1e-13]
    assert tail and all(c <= 10.0 * a * a for a, c in tail)
    _, nrm = o.newton_residual(S)
    assert nrm < 1e-10
    # the wall values of the state (inhomogeneous boundary conditions) are untouched
    wall = np.zeros(S.shape, dtype=bool)
    wall[3, :, :, 0] = wall[3, :, :, -1] = True  # the isothermal walls x = 0, 1 of Theta
    assert np.array_equal(S[wall], S0[wall])


# --- Chebyshev-preconditioned Arnoldi (Section 3.1, the eigenvalue problem Eq (10)) ------------
chebyshev_filter = _solvers.chebyshev_filter
enclosing_ellipse = _solvers.enclosing_ellipse
arnoldi_chebyshev = _solvers.arnoldi_chebyshev


@pytest.mark.parametrize("c2", [2.25, -0.81])
def test_chebyshev_filter_equals_polynomial_ratio(c2):
    """On A = diag(l_i) the filter multiplies component i by T_k((l_i - d)/c) / T_k((lam - d)/c);
    the ratio is evaluated here with numpy's Chebyshev series in complex arithmetic (c imaginary
    when c2 < 0), independently of the real three-term recurrence."""
    rng = np.random.default_rng(6)
    lam_i = np.concatenate([[1.5], -3.0 + 2.5 * rng.random(30)])
    v = rng.standard_normal(31)
    d, lam, k = -1.7, 1.5, 9
    y = chebyshev_filter(lambda x: lam_i * x, v, k, d, c2, lam)
    c = np.sqrt(complex(c2))
    Tk = np.polynomial.chebyshev.Chebyshev.basis(k)
    ratio = Tk((lam_i - d) / c) / Tk((lam - d) / c)
    assert np.max(np.abs(ratio.imag)) < 1e-12 * np.max(np.abs(ratio))
    assert np.allclose(y, ratio.real * v, rtol=1e-11, atol=1e-13)
    assert abs(y[0] - v[0]) < 1e-12 * abs(v[0])  # normalised at lam


def test_enclosing_ellipse_contains_points():
    rng = np.random.default_rng(7)
    pts = -2.0 + rng.standard_normal(40) + 1j * rng.standard_normal(40) * 3.0
    pts = np.concatenate([pts, pts.conj()])
    d, c2 = enclosing_ellipse(pts)
    # the ellipse with foci d +- c (c imaginary when c2 < 0) contains z iff the distances to the
    # foci sum to at most twice its major semi-axis; semi-axes recovered from the points' extent
    re, im = pts.real, np.abs(pts.imag)
    assert abs(d - 0.5 * (re.max() + re.min())) < 1e-12
    a0, b0 = 0.5 * (re.max() - re.min()), im.max()
    s = np.max(((re - d) / a0) ** 2 + (im / b0) ** 2)
    assert abs(c2 - s * (a0 * a0 - b0 * b0)) < 1e-9 * s * (a0 * a0 + b0 * b0)
    c = np.sqrt(complex(c2))
    major = np.sqrt(s) * max(a0, b0)
    assert np.all(np.abs(pts - d - c) + np.abs(pts - d + c) <= 2 * major * (1 + 1e-12))
    assert np.max(np.abs(pts - d - c) + np.abs(pts - d + c)) > 2 * major * (1 - 1e-9)  # and touches


def _dense_with_spectrum(blocks, rest, seed):
    """A real matrix S D S^-1 with D = diag(2x2 rotation blocks for complex pairs, real rest)."""
    rng = np.random.default_rng(seed)
    n = 2 * len(blocks) + len(rest)
    D = np.zeros((n, n))
    for q, (re, im) in enumerate(blocks):
        D[2 * q:2 * q + 2, 2 * q:2 * q + 2] = [[re, im], [-im, re]]
    for i, lam in enumerate(rest):
        D[2 * len(blocks) + i, 2 * len(blocks) + i] = lam
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    S = Q @ np.diag(1.0 + 0.2 * rng.random(n))
    return S @ D @ np.linalg.inv(S), rng.standard_normal(n)


def test_arnoldi_chebyshev_finds_rightmost_complex_pair():
    rng = np.random.default_rng(8)
    A, v0 = _dense_with_spectrum([(-0.1, 2.0), (-1.5, 3.0)], -1.0 - 4.0 * rng.random(196), 8)
    theta, res, info = arnoldi_chebyshev(lambda x: A @ x, v0, 20, 2, 15, 1e-10, 30)
    assert info["converged"] and len(theta) == 2 and info["ellipses"]
    assert np.allclose(sorted(theta, key=lambda z: z.imag), [-0.1 - 2.0j, -0.1 + 2.0j], atol=1e-9)


def test_arnoldi_chebyshev_rightmost_real_with_complex_cloud():
    """Rightmost eigenvalue real, the unwanted ones a complex cloud taller than wide (c2 < 0)."""
    rng = np.random.default_rng(9)
    blocks = [(-2.0 - rng.random(), 1.0 + 5.0 * rng.random()) for _ in range(60)]
    A, v0 = _dense_with_spectrum(blocks, [-0.3, -2.5, -2.8], 9)
    theta, res, info = arnoldi_chebyshev(lambda x: A @ x, v0, 25, 1, 20, 1e-10, 40)
    assert info["converged"] and abs(theta[0] - (-0.3)) < 1e-9
    assert any(c2 < 0 for _, c2 in info["ellipses"])


def test_arnoldi_chebyshev_matches_dense_spectrum_of_krylov_map():
    """The rightmost eigenvalues of the Krylov map on its range (the space of Krylov vectors),
    from a dense eigen-decomposition of the map restricted to an orthonormal basis of that range,
    against the Chebyshev-preconditioned Arnoldi iteration (4^3, CC, Gr = 1e4)."""
    n = (4, 4, 4)
    o = Oracle(*n, gr=1e4)
    S = np.stack(synth.base_flow(*n, synth.CC, 41))
    N = 4 * int(np.prod([m + 2 for m in n]))
    M = np.zeros((N, N))
    for i in range(N):
        e = np.zeros(N)
        e[i] = 1.0
        M[:, i] = o.krylov_vector(S, e.reshape((4,) + o.shape)).ravel()
    U, sv, _ = np.linalg.svd(M)
    Q = U[:, sv > 1e-10 * sv[0]]
    ev = np.linalg.eigvals(Q.T @ M @ Q)
    ev = ev[np.argsort(-ev.real, kind="stable")]
    v0 = o.krylov_vector(S, synth.krylov_input(*n, 3)[0])
    theta, res, info = arnoldi_chebyshev(lambda x: o.krylov_vector(S, x), v0, 30, 1, 12, 1e-10, 60)
    assert info["converged"] and len(theta) == 1
    assert abs(theta[0] - ev[0]) < 1e-8 * max(1.0, abs(ev[0]))


def conduction_leading_eigenvalue(n, gr, pr):
    """U = 0, Theta = 0: the map is block-triangular (T drives v through buoyancy, v does not drive
    T), so its eigenvalues are those of kappa times the temperature Laplacian with the homogeneous
    BCs (Kronecker sums of 1D eigenvalues, Eq (17)) and those of the Stokes block. With Pr = 10 the
    slowest temperature mode decays far more slowly than the slowest Stokes mode, so the leading
    eigenvalue is kappa times the sum of the largest 1D Dirichlet eigenvalues (wall nodes on the
    walls: the first and last cells see a half spacing)."""
    kappa = 1 / (pr * gr ** 0.5)

    def largest_dirichlet_1d(m):
        h = 1.0 / m
        M = np.zeros((m, m))
        for t in range(m):
            wl = 2.0 if t == 0 else 1.0
            wr = 2.0 if t == m - 1 else 1.0
            M[t, t] = -(wl + wr) / h ** 2
            if t > 0:
                M[t, t - 1] = 1 / h ** 2
            if t < m - 1:
                M[t, t + 1] = 1 / h ** 2
        return np.linalg.eigvalsh(M).max()

    return kappa * sum(largest_dirichlet_1d(m) for m in n)


def test_arnoldi_chebyshev_conduction_closed_form():
    n, gr, pr = (5, 6, 4), 1e6, 10.0
    o = Oracle(*n, gr=gr, pr=pr)
    base = np.zeros((4,) + o.shape)
    v0 = o.krylov_vector(base, synth.krylov_input(*n, 5)[0])
    theta, res, info = arnoldi_chebyshev(lambda x: o.krylov_vector(base, x), v0, 30, 1, 12, 1e-11, 60)
    lead = conduction_leading_eigenvalue(n, gr, pr)
    assert info["converged"] and len(theta) == 1
    assert abs(theta[0] - lead) < 1e-9 * abs(lead)
