"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names the passage of arXiv 1905.11601 it checks. They run on CPU only.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import Oracle
from paper_1905_11601_gb300 import synth
from tests.mac_assembly import MacOps
from tests.oracle_helpers import project_output_side

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def packed_base(nx, ny, nz, bc, seed):
    return np.stack(synth.base_flow(nx, ny, nz, bc, seed))


def rand_vec(nx, ny, nz, seed):
    return synth.krylov_input(nx, ny, nz, seed)[0]


def mac_div(vel, n):
    """Divergence of a packed velocity on the interior cells, written with numpy slices."""
    nx, ny, nz = n
    u, v, w = vel
    return ((u[1:-1, 1:-1, 1:-1] - u[1:-1, 1:-1, :-2]) * nx + (v[1:-1, 1:-1, 1:-1] - v[1:-1, :-2, 1:-1]) * ny
            + (w[1:-1, 1:-1, 1:-1] - w[:-2, 1:-1, 1:-1]) * nz)


GRIDS = [(4, 4, 4), (5, 4, 6), (7, 6, 5)]


# --- Eq (15): 1D eigen-decomposition of the Neumann Laplacian --------------------------------
@pytest.mark.parametrize("n", [2, 3, 8, 17])
def test_neumann_eigenpairs_match_library_eigensolver(n):
    o = Oracle(n, 3, 3)
    h = 1.0 / n
    # D G on one axis with the wall faces excluded: (D v)_t = (v_t - v_{t-1})/h, v_0 = v_n = 0
    Dm = np.zeros((n, n - 1))
    for t in range(n):
        if t < n - 1:
            Dm[t, t] = 1.0 / h
        if t > 0:
            Dm[t, t - 1] = -1.0 / h
    L = -Dm @ Dm.T
    E, Einv, lam = o.axis_data(0, 0), o.axis_data(0, 1), o.axis_data(0, 2)
    assert np.allclose(L @ E, E * lam[None, :], atol=1e-9 / h ** 2 * 1e-3)
    assert np.allclose(Einv @ E, np.eye(n), atol=1e-13)
    assert np.allclose(np.sort(lam), np.sort(np.linalg.eigvalsh(L)), rtol=1e-12, atol=1e-9)
    assert abs(lam[0]) < 1e-12  # the Neumann zero mode


# --- Eq (18): TPD Poisson equals a dense solve of the assembled operator ----------------------
@pytest.mark.parametrize("n", GRIDS)
def test_tpd_poisson_matches_dense_solve(n):
    nx, ny, nz = n
    o = Oracle(nx, ny, nz)
    ops = MacOps(nx, ny, nz)
    DG = (ops.divergence() @ ops.gradient()).toarray()
    cm = ops.dof_mask(3).astype(bool)
    A = DG[np.ix_(cm, cm)]
    rng = np.random.default_rng(3)
    b = rng.standard_normal(nx * ny * nz)
    b -= b.mean()  # compatibility of the Neumann problem
    phi_dense = np.linalg.lstsq(A, b, rcond=None)[0]
    phi_dense -= phi_dense.mean()
    phi = o.poisson(b.reshape(nz, ny, nx)).ravel()
    assert abs(phi.mean()) < 1e-13
    assert np.allclose(phi, phi_dense, rtol=0, atol=1e-12 * np.abs(phi_dense).max())
    assert np.linalg.norm(A @ phi - b) < 1e-12 * np.linalg.norm(b)


# --- Eqs (19)-(21): temperature projection ---------------------------------------------------
@pytest.mark.parametrize("bc", [synth.CC, synth.AA])
def test_temperature_projection_is_orthogonal_projector_onto_bc_space(bc):
    n = (5, 6, 4)
    o = Oracle(*n, bc=bc)
    for a in range(3):
        Pa = o.axis_data(a, 3)
        m = Pa.shape[0]
        assert np.allclose(Pa @ Pa, Pa, atol=1e-13)
        assert np.allclose(Pa, Pa.T, atol=1e-13)
        # the BC subspace: Dirichlet walls 0; insulated walls equal to the neighbour
        if a == 1 and bc == synth.AA:
            basis = np.zeros((m, m - 2))
            for t in range(1, m - 1):
                basis[t, t - 1] = 1.0
            basis[0, 0] = 1.0
            basis[m - 1, m - 3] = 1.0
        else:
            basis = np.eye(m)[:, 1:m - 1]
        Q = sla.orth(basis)
        assert np.allclose(Pa, Q @ Q.T, atol=1e-13)


@pytest.mark.parametrize("bc", [synth.CC, synth.AA])
def test_gram_form_equals_closed_form(bc):
    n = (5, 6, 4)
    o = Oracle(*n, bc=bc)
    T = rand_vec(*n, seed=5)[3]
    g = o.tproj_gram(T)
    c = o.tproj_closed(T)
    assert np.allclose(g, c, rtol=0, atol=1e-14)


@pytest.mark.parametrize("bc,tproj", [(synth.CC, 0), (synth.AA, 0), (synth.AA, 1)])
def test_projected_temperature_satisfies_bcs_exactly(bc, tproj):
    n = (6, 5, 7)
    o = Oracle(*n, bc=bc, tproj=tproj)
    base = packed_base(*n, bc, 9)
    y = o.krylov_vector(base, rand_vec(*n, 10))
    T = y[3]
    # Eq (4), Eq (5) homogeneous: Dirichlet on x and z walls, bitwise zero
    assert np.all(T[:, :, 0] == 0) and np.all(T[:, :, -1] == 0)
    assert np.all(T[0] == 0) and np.all(T[-1] == 0)
    if bc == synth.CC:  # Eq (6)
        assert np.all(T[:, 0, :] == 0) and np.all(T[:, -1, :] == 0)
    else:  # Eq (7), discrete: wall node equals its neighbour
        assert np.array_equal(T[:, 0, :], T[:, 1, :])
        assert np.array_equal(T[:, -1, :], T[:, -2, :])


# --- Section 3.1: the SIMPLE / Chorin velocity projection -------------------------------------
@pytest.mark.parametrize("n", GRIDS + [(16, 16, 16)])
def test_velocity_divergence_free_after_projection(n):
    o = Oracle(*n)
    base = packed_base(*n, synth.CC, 4)
    y, st = o.krylov_vector(base, rand_vec(*n, 11), stats=True)
    div = mac_div(y[:3], n)
    vmax = np.abs(y[:3]).max()
    assert np.abs(div).max() * (1.0 / max(n)) / vmax < 1e-13
    # SIMPLE converged in fewer than 10 passes (the paper's statement)
    figures = json.load(open(os.path.join(GOLDEN, "paper_figures.json")))
    assert st.passes < figures["simple_passes_upper_bound"]["value"]
    # wall-normal faces and tangential wall nodes are zero (no-slip, Eq (13))
    ops = MacOps(*n)
    for F in range(3):
        mask = ops.dof_mask(F).reshape(y[F].shape).astype(bool)
        assert np.all(y[F][~mask] == 0)


def _pi_v(o, ops, vel):
    b = o.divergence(vel)
    phi = o.poisson(b)
    out, _ = o.correct(phi, vel)
    return out


def test_velocity_projection_is_orthogonal_and_keeps_curls():
    n = (5, 6, 4)
    nx, ny, nz = n
    o = Oracle(*n)
    ops = MacOps(*n)
    rng = np.random.default_rng(1)
    masks = [ops.dof_mask(F).reshape(o.shape).astype(bool) for F in range(3)]

    def rv():
        v = rng.standard_normal((3,) + o.shape)
        for F in range(3):
            v[F][~masks[F]] = 0
        return v

    a, b = rv(), rv()
    pa, pb = _pi_v(o, ops, a), _pi_v(o, ops, b)
    assert np.allclose(_pi_v(o, ops, pa), pa, atol=1e-12)
    assert abs(np.vdot(a, pb) - np.vdot(pa, b)) < 1e-12 * np.linalg.norm(a) * np.linalg.norm(b)
    # discrete curl of a potential vanishing on the walls is divergence-free: Pi keeps it
    U, V, W = synth.base_velocity(nx, ny, nz, np.random.default_rng(2))
    c = np.stack([U, V, W])
    assert np.allclose(_pi_v(o, ops, c), c, atol=1e-14)
    # gradients are removed entirely
    phi = rng.standard_normal((nz, ny, nx))
    g = (ops.gradient() @ np.pad(phi, 1).ravel()).reshape((3,) + o.shape)
    assert np.abs(_pi_v(o, ops, g)).max() < 1e-10 * np.abs(g).max()


def test_simple_second_pass_changes_nothing():
    n = (6, 6, 6)
    base = packed_base(*n, synth.CC, 2)
    x = rand_vec(*n, 3)
    y1, st1 = Oracle(*n).krylov_vector(base, x, stats=True)
    o3 = Oracle(*n, tol=0.0, max_passes=3)
    y3, st3 = o3.krylov_vector(base, x, stats=True)
    assert st1.passes == 1 and st3.passes == 3
    assert np.allclose(y1, y3, rtol=0, atol=1e-12 * np.abs(y1).max())


# --- Eqs (8)-(9), (11)-(12): the linearised operator --------------------------------------------
@pytest.mark.parametrize("n,bc", [((4, 4, 4), synth.CC), ((5, 4, 6), synth.CC), ((5, 4, 6), synth.AA)])
def test_jacobian_matches_kronecker_assembly(n, bc):
    o = Oracle(*n, bc=bc, gr=2.0e6, pr=0.71)
    base = packed_base(*n, bc, 21)
    xp = o.project_input(rand_vec(*n, 22))
    J = MacOps(*n).jacobian(base, 2.0e6, 0.71)
    y_asm = (J @ xp.ravel()).reshape(xp.shape)
    y_or = o.jx_raw(base, xp)
    assert np.allclose(y_or, y_asm, rtol=0, atol=1e-12 * np.abs(y_asm).max())


def _linear(coef, Z, Y, X):
    return coef[0] + coef[1] * X + coef[2] * Y + coef[3] * Z


def _coords(n, F):
    nx, ny, nz = n
    xs = [synth.face_coords(nx) if F == 0 else synth.cell_coords(nx),
          synth.face_coords(ny) if F == 1 else synth.cell_coords(ny),
          synth.face_coords(nz) if F == 2 else synth.cell_coords(nz)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return Z, Y, X


def test_advection_exact_for_linear_fields_in_the_interior():
    """Central differences and midpoint averages are exact for linear fields."""
    n = (8, 7, 9)
    gr, pr = 1.0e6, 0.71
    o = Oracle(*n, gr=gr, pr=pr)
    rng = np.random.default_rng(5)
    cb = rng.standard_normal((4, 4))
    cx = rng.standard_normal((4, 4))
    base = np.stack([_linear(cb[F], *_coords(n, F)) for F in range(4)])
    x = np.stack([_linear(cx[F], *_coords(n, F)) for F in range(4)])
    y = o.jx_raw(base, x)  # x used as given: no projection, so interior rows see linear data
    grad = lambda c: c[1:]  # noqa: E731  (d/dx, d/dy, d/dz of a linear field)
    for F in range(4):
        Z, Y, X = _coords(n, F)
        ub = [_linear(cb[c], Z, Y, X) for c in range(3)]
        ux = [_linear(cx[c], Z, Y, X) for c in range(3)]
        if F == 3:
            exact = -sum(ub[c] * grad(cx[3])[c] for c in range(3)) - sum(ux[c] * grad(cb[3])[c] for c in range(3))
        else:
            exact = -sum(ub[c] * grad(cx[F])[c] for c in range(3)) - sum(ux[c] * grad(cb[F])[c] for c in range(3))
            if F == 2:
                exact = exact + _linear(cx[3], Z, Y, X)
        sl = (slice(2, -2),) * 3
        assert np.allclose(y[F][sl], exact[sl], rtol=0, atol=1e-11), F


def test_diffusion_exact_for_quadratics_in_the_interior():
    n = (8, 8, 8)
    gr, pr = 1.0e6, 0.71
    o = Oracle(*n, gr=gr, pr=pr)
    base = np.zeros((4,) + o.shape)
    x = np.zeros((4,) + o.shape)
    for F in range(4):
        Z, Y, X = _coords(n, F)
        x[F] = X ** 2 + 2 * Y ** 2 - 0.5 * Z ** 2 + X * Y
    y = o.jx_raw(base, x)
    lap = 2 + 4 - 1.0
    sl = (slice(2, -2),) * 3
    for F in range(3):
        expect = gr ** -0.5 * lap + (0.5 * (x[3][:-1] + x[3][1:]) if F == 2 else 0)
        if F == 2:
            expect = np.concatenate([expect, np.zeros((1,) + o.shape[1:])])
        assert np.allclose(y[F][sl], np.broadcast_to(expect, y[F].shape)[sl], rtol=0, atol=1e-10)
    assert np.allclose(y[3][sl], lap / (pr * gr ** 0.5), rtol=0, atol=1e-10)


def _centro(vec):
    """S3 of Section 2 on a packed field: {u,v,w,theta}(x) -> -{u,v,w,theta}(1-x).

    Cell-like index t maps to n+1-t; face-like index t maps to n-t (padding stays put)."""
    out = np.zeros_like(vec)
    for F in range(4):
        f = vec[F]
        g = f[::-1, ::-1, ::-1]  # cell-like reversal on all axes
        if F < 3:
            # along the face axis the map is t -> n - t: reverse then shift by one
            g = np.roll(g, -1, axis=2 - F)
        out[F] = -g
    # face padding (index n+1) must stay zero
    for F in range(3):
        idx = [slice(None)] * 3
        idx[2 - F] = -1
        out[F][tuple(idx)] = 0.0
    return out


def test_jacobian_commutes_with_centro_symmetry():
    """Section 2, symmetry (iii): a centro-symmetric base flow makes J commute with S3."""
    n = (6, 5, 7)
    o = Oracle(*n)
    b = packed_base(*n, synth.CC, 31)
    theta = b[3].copy()
    Z, Y, X = _coords(n, 3)
    lin = 1 - X
    th = theta - lin
    bs = b.copy()
    bs[3] = th
    bs = 0.5 * (bs + _centro(bs))
    bs[3] = bs[3] + lin
    xp = o.project_input(rand_vec(*n, 32))
    y1 = _centro(o.jx_raw(bs, xp))
    y2 = o.jx_raw(bs, _centro(xp))
    assert np.allclose(y1, y2, rtol=0, atol=1e-12 * np.abs(y1).max())


@pytest.mark.parametrize("n", [(4, 5, 3), (3, 3, 6)])
def test_conduction_spectrum_is_kronecker_sum(n):
    """U = 0, Theta = 0: the temperature block is kappa times the Laplacian with the
    homogeneous BCs, whose eigenvalues are the sums of 1D eigenvalues (Eq 17)."""
    nx, ny, nz = n
    gr, pr = 1.0e6, 0.71
    kappa = 1 / (pr * gr ** 0.5)
    o = Oracle(*n, gr=gr, pr=pr)
    base = np.zeros((4,) + o.shape)
    cols = []
    for k in range(1, nz + 1):
        for j in range(1, ny + 1):
            for i in range(1, nx + 1):
                x = np.zeros((4,) + o.shape)
                x[3, k, j, i] = 1.0
                cols.append(o.krylov_vector(base, x)[3, 1:-1, 1:-1, 1:-1].ravel())
    A = np.array(cols).T
    ev = np.sort(np.linalg.eigvals(A).real)

    def dirichlet_1d(m):
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
        return np.linalg.eigvalsh(M)

    lx, ly, lz = dirichlet_1d(nx), dirichlet_1d(ny), dirichlet_1d(nz)
    expect = np.sort((kappa * (lz[:, None, None] + ly[None, :, None] + lx[None, None, :])).ravel())
    assert np.allclose(ev, expect, rtol=1e-10)


# --- Newton step 2 and the Jacobian: F is quadratic, so central differences are exact ----------
@pytest.mark.parametrize("bc", [synth.CC, synth.AA])
def test_finite_difference_of_residual_equals_krylov_vector(bc):
    n = (6, 7, 5)
    o = Oracle(*n, bc=bc, gr=2.0e6)
    S = packed_base(*n, bc, 41)
    x = o.project_input(rand_vec(*n, 42))
    eps = 1e-3
    Fp, _ = o.newton_residual(S + eps * x)
    Fm, _ = o.newton_residual(S - eps * x)
    fd = (Fp - Fm) / (2 * eps)
    y = o.krylov_vector(S, x)
    assert np.linalg.norm(fd - y) < 1e-10 * np.linalg.norm(y)


# --- Arnoldi (Sections 3.1 / 4): A V_k = V_{k+1} H, orthonormal basis ----------------------------
def test_arnoldi_relation_and_orthonormality():
    n = (6, 6, 6)
    o = Oracle(*n, gr=1e6)
    base = packed_base(*n, synth.CC, 51)
    k = 8
    V = np.zeros((k + 1, 4) + o.shape)
    v0 = o.project_input(rand_vec(*n, 52))
    V[0] = v0 / np.linalg.norm(v0)
    H = np.zeros((k + 1, k))
    for j in range(k):
        H[: j + 2, j] = o.arnoldi_step(base, V, j)
    Vm = V.reshape(k + 1, -1)
    assert np.abs(Vm @ Vm.T - np.eye(k + 1)).max() < 1e-13
    AV = np.stack([o.krylov_vector(base, V[j]) for j in range(k)]).reshape(k, -1)
    assert np.linalg.norm(AV.T - Vm.T @ H) < 1e-12 * np.linalg.norm(AV)


# --- the transpose of the Krylov map and the base-flow gradient (adjoint eigenmodes, sensitivity) --
@pytest.mark.parametrize("n,bc", [((6, 5, 7), synth.CC), ((5, 6, 4), synth.AA)])
def test_adjoint_dot_product(n, bc):
    """<y, J x> = <J^T y, x> and <y, A x> = <A^T y, x> (the definition of the transpose)."""
    o = Oracle(*n, bc=bc, gr=2e6)
    base = packed_base(*n, bc, 71)
    x = synth.krylov_input(*n, 72, 2)
    xp = o.project_input(x[0])
    lhs, rhs = np.vdot(x[1], o.jx_raw(base, xp)), np.vdot(o.jt_raw(base, x[1]), xp)
    assert abs(lhs - rhs) < 1e-13 * np.linalg.norm(x[1]) * np.linalg.norm(o.jx_raw(base, xp))
    A = o.krylov_vector(base, x[0])
    lhs, rhs = np.vdot(x[1], A), np.vdot(o.krylov_adjoint(base, x[1]), x[0])
    assert abs(lhs - rhs) < 1e-13 * np.linalg.norm(x[1]) * np.linalg.norm(A)


def test_jt_matches_transpose_of_kronecker_assembly():
    n = (5, 4, 6)
    o = Oracle(*n, gr=2e6)
    base = packed_base(*n, synth.CC, 73)
    ys = rand_vec(*n, 74)
    J = MacOps(*n).jacobian(base, 2e6, 0.71)
    z_asm = (J.T @ ys.ravel()).reshape(ys.shape)
    z = o.jt_raw(base, ys)
    assert np.allclose(z, z_asm, rtol=0, atol=1e-12 * np.abs(z_asm).max())


@pytest.mark.parametrize("bc", [synth.CC, synth.AA])
def test_base_gradient_matches_central_differences(bc):
    """<y, J(b) x> is affine in the base state b, so a central difference is exact up to rounding."""
    n = (6, 5, 4)
    o = Oracle(*n, bc=bc, gr=2e6)
    base = packed_base(*n, bc, 75)
    x = synth.krylov_input(*n, 76, 2)
    xp, ys = o.project_input(x[0]), x[1]
    g = o.grad_base(xp, ys)
    rng = np.random.default_rng(77)
    for _ in range(3):
        d = rng.standard_normal(base.shape)
        h = 1e-3
        fp = np.vdot(ys, o.jx_raw(base + h * d, xp))
        fm = np.vdot(ys, o.jx_raw(base - h * d, xp))
        assert abs((fp - fm) / (2 * h) - np.vdot(g, d)) < 1e-10 * abs(np.vdot(g, d)) + 1e-12
    # entries no stencil reads (edges and corners of the padded box) have zero gradient
    assert np.all(g[:, 0, 0, :] == 0) and np.all(g[:, -1, :, 0] == 0)


def test_grashof_derivative_matches_central_differences():
    n = (5, 5, 6)
    base = packed_base(*n, synth.CC, 78)
    x = synth.krylov_input(*n, 79, 2)
    gr, h = 2e6, 1e2
    o = Oracle(*n, gr=gr)
    xp, ys = o.project_input(x[0]), x[1]
    d = o.grad_gr(xp, ys)
    fp = np.vdot(ys, Oracle(*n, gr=gr + h).jx_raw(base, xp))
    fm = np.vdot(ys, Oracle(*n, gr=gr - h).jx_raw(base, xp))
    assert abs((fp - fm) / (2 * h) - d) < 1e-6 * abs(d)


def test_rayleigh_quotient_gradient_in_theta():
    """R = <y, A x> / <y, x>: its gradient in Theta is grad_base(P_BC x, (Pi (+) P_T) y) / <y, x>,
    checked against central differences with h = 1e-6."""
    n = (6, 6, 5)
    o = Oracle(*n, gr=2e6)
    base = packed_base(*n, synth.CC, 80)
    x = synth.krylov_input(*n, 81, 2)
    yx = np.vdot(x[1], x[0])
    R = lambda b: np.vdot(x[1], o.krylov_vector(b, x[0])) / yx  # noqa: E731
    xp = o.project_input(x[0])
    yhat = project_output_side(o, x[1])  # the (symmetric) output projections of A applied to y
    gb = o.grad_base(xp, yhat) / yx
    d = np.zeros_like(base)
    d[3] = np.random.default_rng(82).standard_normal(base.shape[1:])
    h = 1e-6
    fd = (R(base + h * d) - R(base - h * d)) / (2 * h)
    assert abs(fd - np.vdot(gb, d)) < 1e-7 * abs(np.vdot(gb, d))
