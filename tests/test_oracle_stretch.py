"""Pins of the FP64 oracle on stretched grids (Eq 22, Section 3.2) against facts that do not
come from the oracle: the closed form of the mapping, an independent Kronecker assembly of the
operators, the finite-volume conservation identity, exactness of the 3-point derivative for
quadratics, the self-adjointness of the velocity projection in the volume-weighted product,
second-order convergence of the Poisson solve, and the uniform limit. CPU only."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1905_11601_gb300 import synth
from tests.mac_assembly import MacOps, control_volume, positions, stretched_faces

S = 0.12  # the steepest stretching used in Section 3.2
GRIDS = [(4, 4, 4), (5, 4, 6), (7, 6, 5)]


def packed_base(nx, ny, nz, bc, seed):
    return np.stack(synth.base_flow(nx, ny, nz, bc, seed))


def rand_vec(nx, ny, nz, seed):
    return synth.krylov_input(nx, ny, nz, seed)[0]


def cell_widths(n, s):
    return np.diff(stretched_faces(n, s))


def cell_volumes(n, s):
    """Compact (nz, ny, nx) array of cell volumes."""
    dx, dy, dz = (cell_widths(m, s) for m in n)
    return dz[:, None, None] * dy[None, :, None] * dx[None, None, :]


def face_volumes(n, s, shape):
    """Padded (3, nz+2, ny+2, nx+2) control volumes of the u, v, w faces (interior rows)."""
    out = np.zeros((3,) + shape)
    for F in range(3):
        w = [control_volume(n[a], F == a, s) for a in range(3)]
        out[F] = w[2][:, None, None] * w[1][None, :, None] * w[0][None, None, :]
    return out


# --- Eq (22): the mapping -------------------------------------------------------------------------
def test_face_coordinates_follow_eq22():
    n = 16
    o = Oracle(n, 8, 12, stretch=S)
    xf, xc = o.axis_data(0, 4), o.axis_data(0, 5)
    assert xf[0] == 0.0 and xf[-1] == 1.0 and np.all(np.diff(xf) > 0)
    # sin(2 pi xi) = 1, 0, -1 at xi = 1/4, 1/2, 3/4
    assert abs(xf[n // 4] - (0.25 - S)) < 1e-15
    assert abs(xf[n // 2] - 0.5) < 1e-15
    assert abs(xf[3 * n // 4] - (0.75 + S)) < 1e-15
    assert np.allclose(xf + xf[::-1], 1.0, rtol=0, atol=2e-16)  # mirror symmetry about 1/2
    assert xc[0] == 0.0 and xc[-1] == 1.0
    assert np.array_equal(xc[1:-1], 0.5 * (xf[:-1] + xf[1:]))
    # the wall cell: dx/dxi = 1 - 2 pi s at the walls, up to the Taylor remainder
    assert abs((xf[1] - xf[0]) * n - (1 - 2 * np.pi * S)) <= S * (2 * np.pi) ** 3 / (6 * n * n)
    # s = 0 is the uniform grid
    u = Oracle(n, 8, 12)
    assert np.allclose(u.axis_data(0, 4), np.arange(n + 1) / n, rtol=0, atol=1e-16)


def test_invalid_stretch_is_rejected():
    for s in (-0.01, 0.5 / np.pi, 0.2):
        with pytest.raises(ValueError):
            Oracle(4, 4, 4, stretch=s)


# --- Eqs (8)-(9), (11)-(12) on the stretched grid ------------------------------------------------
@pytest.mark.parametrize("n,bc", [((4, 4, 4), synth.CC), ((5, 4, 6), synth.CC), ((5, 4, 6), synth.AA),
                                  ((7, 6, 5), synth.AA)])
def test_stretched_jacobian_matches_kronecker_assembly(n, bc):
    o = Oracle(*n, bc=bc, gr=2.0e6, pr=0.71, stretch=S)
    base = packed_base(*n, bc, 21)
    xp = o.project_input(rand_vec(*n, 22))
    J = MacOps(*n, s=S).jacobian(base, 2.0e6, 0.71)
    y_asm = (J @ xp.ravel()).reshape(xp.shape)
    y_or = o.jx_raw(base, xp)
    assert np.allclose(y_or, y_asm, rtol=0, atol=1e-12 * np.abs(y_asm).max())


def test_diffusion_conserves_flux():
    """Finite-volume identity: the volume-weighted sum of the flux-form Laplacian over the
    control volumes telescopes to the fluxes through the walls."""
    n = (6, 5, 7)
    nx, ny, nz = n
    o = Oracle(*n, gr=1.0, pr=1.0, stretch=S)  # nu = kappa = 1
    rng = np.random.default_rng(8)
    x = rng.standard_normal((4,) + o.shape)
    y = o.jx_raw(np.zeros_like(x), x)
    # temperature: every cell is a control volume; wall nodes at 0 and 1
    T = x[3]
    c = [positions(m, False, S) for m in n]
    dx, dy, dz = (cell_widths(m, S) for m in n)
    lhs = np.sum(cell_volumes(n, S) * y[3][1:-1, 1:-1, 1:-1])
    Ti = T[1:-1, 1:-1, 1:-1]
    fx = (T[1:-1, 1:-1, -1] - Ti[:, :, -1]) / (1 - c[0][nx]) - (Ti[:, :, 0] - T[1:-1, 1:-1, 0]) / c[0][1]
    fy = (T[1:-1, -1, 1:-1] - Ti[:, -1, :]) / (1 - c[1][ny]) - (Ti[:, 0, :] - T[1:-1, 0, 1:-1]) / c[1][1]
    fz = (T[-1, 1:-1, 1:-1] - Ti[-1]) / (1 - c[2][nz]) - (Ti[0] - T[0, 1:-1, 1:-1]) / c[2][1]
    rhs = (np.sum(fx * dz[:, None] * dy[None, :]) + np.sum(fy * dz[:, None] * dx[None, :])
           + np.sum(fz * dy[:, None] * dx[None, :]))
    assert abs(lhs - rhs) < 1e-12 * np.sum(np.abs(cell_volumes(n, S) * y[3][1:-1, 1:-1, 1:-1]))
    # u: faces 1..nx-1 along x (control volumes between cell centres), cells along y and z
    u = x[0]
    vol = face_volumes(n, S, o.shape)[0]
    ui = u[1:-1, 1:-1, 1:nx]
    lhs = np.sum(vol[1:-1, 1:-1, 1:nx] * y[0][1:-1, 1:-1, 1:nx])
    gx = (u[1:-1, 1:-1, nx] - u[1:-1, 1:-1, nx - 1]) / dx[-1] - (u[1:-1, 1:-1, 1] - u[1:-1, 1:-1, 0]) / dx[0]
    gxc = control_volume(nx, True, S)[1:nx]
    gy = (u[1:-1, -1, 1:nx] - ui[:, -1, :]) / (1 - c[1][ny]) - (ui[:, 0, :] - u[1:-1, 0, 1:nx]) / c[1][1]
    gz = (u[-1, 1:-1, 1:nx] - ui[-1]) / (1 - c[2][nz]) - (ui[0] - u[0, 1:-1, 1:nx]) / c[2][1]
    rhs = (np.sum(gx * dz[:, None] * dy[None, :]) + np.sum(gy * dz[:, None] * gxc[None, :])
           + np.sum(gz * dy[:, None] * gxc[None, :]))
    assert abs(lhs - rhs) < 1e-12 * np.sum(np.abs(vol[1:-1, 1:-1, 1:nx] * y[0][1:-1, 1:-1, 1:nx]))


def test_advection_exact_for_quadratics():
    """The 3-point derivative on the non-uniform nodes is exact for quadratics; with a constant
    base state the interpolated velocities are exact too (diffusion made negligible)."""
    n = (9, 8, 10)
    gr = 1.0e30
    o = Oracle(*n, gr=gr, pr=1.0, stretch=S)
    Ub = np.array([0.7, -0.4, 0.9, 0.3])
    base = np.stack([np.full(o.shape, Ub[F]) for F in range(4)])
    coords = []
    for F in range(4):
        xs = [positions(n[a], F == a, S) for a in range(3)]
        coords.append(np.meshgrid(xs[2], xs[1], xs[0], indexing="ij"))
    q = [(1.0, -2.0, 0.5), (0.3, 1.1, -0.8), (-1.2, 0.4, 2.0), (0.6, 0.9, -1.5)]
    x = np.stack([q[F][0] * coords[F][2] ** 2 + q[F][1] * coords[F][1] ** 2 + q[F][2] * coords[F][0] * coords[F][2]
                  for F in range(4)])
    y = o.jx_raw(base, x)
    sl = (slice(2, -2),) * 3
    for F in range(4):
        Z, Y, X = coords[F]
        ddx = 2 * q[F][0] * X + q[F][2] * Z
        ddy = 2 * q[F][1] * Y
        ddz = q[F][2] * X
        expect = -(Ub[0] * ddx + Ub[1] * ddy + Ub[2] * ddz)
        if F == 2:
            expect = expect + np.concatenate([0.5 * (x[3][:-1] + x[3][1:]), np.zeros((1,) + o.shape[1:])])
        assert np.allclose(y[F][sl], expect[sl], rtol=0, atol=1e-11), F


# --- Eqs (14)-(18) on the stretched grid -----------------------------------------------------------
@pytest.mark.parametrize("n", [2, 3, 8, 17])
def test_stretched_neumann_eigenpairs(n):
    o = Oracle(n, 3, 3, stretch=S)
    dx = cell_widths(n, S)
    c = positions(n, False, S)
    g = c[2:n + 1] - c[1:n]
    # D G along one axis from its two factors, the wall faces excluded
    Dm = np.zeros((n, n - 1))
    Gm = np.zeros((n - 1, n))
    for t in range(n - 1):
        Gm[t, t + 1], Gm[t, t] = 1.0 / g[t], -1.0 / g[t]
        Dm[t, t] += 1.0 / dx[t]
        Dm[t + 1, t] -= 1.0 / dx[t + 1]
    A = Dm @ Gm
    E, Einv, lam = o.axis_data(0, 0), o.axis_data(0, 1), o.axis_data(0, 2)
    scale = np.abs(A).max()
    assert np.abs(A @ E - E * lam[None, :]).max() < 1e-12 * scale
    assert np.allclose(Einv @ E, np.eye(n), rtol=0, atol=1e-12)
    assert lam[0] == 0.0 and np.all(np.diff(lam) < 0)
    ref = np.sort(np.linalg.eigvals(A).real)[::-1]
    assert np.allclose(lam[1:], ref[1:], rtol=1e-12, atol=1e-12 * scale)
    assert abs(ref[0]) < 1e-12 * scale
    assert np.allclose(E[:, 0], E[0, 0], rtol=1e-12, atol=0)  # the constant mode


@pytest.mark.parametrize("n", GRIDS)
def test_stretched_tpd_poisson_matches_dense_solve(n):
    nx, ny, nz = n
    o = Oracle(*n, stretch=S)
    ops = MacOps(*n, s=S)
    DG = (ops.divergence() @ ops.gradient()).toarray()
    cm = ops.dof_mask(3).astype(bool)
    A = DG[np.ix_(cm, cm)]
    w = cell_volumes(n, S).ravel()
    rng = np.random.default_rng(3)
    b = rng.standard_normal(nx * ny * nz)
    b -= np.dot(w, b) / w.sum()  # the volume-weighted sum vanishes: the Neumann compatibility
    phi_dense = np.linalg.lstsq(A, b, rcond=None)[0]
    phi_dense -= np.dot(w, phi_dense) / w.sum()
    phi = o.poisson(b.reshape(nz, ny, nx)).ravel()
    assert abs(np.dot(w, phi)) < 1e-13 * np.abs(phi).max()
    assert np.allclose(phi, phi_dense, rtol=0, atol=1e-11 * np.abs(phi_dense).max())
    assert np.linalg.norm(A @ phi - b) < 1e-12 * np.linalg.norm(A, 2) * np.linalg.norm(phi)


def test_stretched_poisson_converges_at_second_order():
    def err(m):
        o = Oracle(m, m, m, stretch=S)
        c = positions(m, False, S)[1:-1]
        Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
        ex = np.cos(np.pi * X) * np.cos(np.pi * Y) * np.cos(np.pi * Z)
        w = cell_volumes((m, m, m), S)
        b = -3 * np.pi ** 2 * ex
        b -= np.sum(w * b) / w.sum()
        phi = o.poisson(b)
        ex = ex - np.sum(w * ex) / w.sum()
        return np.abs(phi - ex).max()

    e1, e2 = err(12), err(24)
    assert e2 < 0.05 and e1 / e2 > 3.0, (e1, e2)


# --- Section 3.1's projection on the stretched grid ------------------------------------------------
@pytest.mark.parametrize("n", GRIDS + [(16, 16, 16)])
def test_stretched_velocity_divergence_free_after_projection(n):
    o = Oracle(*n, stretch=S)
    base = packed_base(*n, synth.CC, 4)
    y, st = o.krylov_vector(base, rand_vec(*n, 11), stats=True)
    D = MacOps(*n, s=S).divergence()
    div = D @ y[:3].ravel()
    hmin = min(cell_widths(m, S).min() for m in n)
    assert np.abs(div).max() * hmin / np.abs(y[:3]).max() < 1e-13
    assert st.passes < 10


def test_projection_is_self_adjoint_in_the_volume_product():
    """Pi_v = I - G (D G)^+ D with D = -W^-1 G^T M (W cell volumes, M face volumes) is an
    M-orthogonal projector: <a, Pi b>_M = <Pi a, b>_M, Pi Pi = Pi, and Pi G phi = 0."""
    n = (5, 6, 4)
    o = Oracle(*n, stretch=S)
    ops = MacOps(*n, s=S)
    rng = np.random.default_rng(1)
    masks = [ops.dof_mask(F).reshape(o.shape).astype(bool) for F in range(3)]
    M = face_volumes(n, S, o.shape)

    def rv():
        v = rng.standard_normal((3,) + o.shape)
        for F in range(3):
            v[F][~masks[F]] = 0
        return v

    def pi(v):
        out, _ = o.correct(o.poisson(o.divergence(v)), v)
        return out

    a, b = rv(), rv()
    pa, pb = pi(a), pi(b)
    na, nb = np.sqrt(np.sum(M * a * a)), np.sqrt(np.sum(M * b * b))
    assert abs(np.sum(M * a * pb) - np.sum(M * pa * b)) < 1e-12 * na * nb
    assert np.allclose(pi(pa), pa, rtol=0, atol=1e-12 * np.abs(pa).max())
    phi = rng.standard_normal(n[::-1])
    g = (ops.gradient() @ np.pad(phi, 1).ravel()).reshape((3,) + o.shape)
    assert np.abs(pi(g)).max() < 1e-10 * np.abs(g).max()


# --- the uniform limit ----------------------------------------------------------------------------
def test_small_stretch_approaches_the_uniform_grid():
    """s = 1e-9 runs the numeric eigen-decomposition and the stretched widths; it must agree
    with the closed-form cosine basis of the uniform grid to O(s)."""
    n = (6, 5, 7)
    base = packed_base(*n, synth.CC, 4)
    x = rand_vec(*n, 9)
    o0, o1 = Oracle(*n), Oracle(*n, stretch=1e-9)
    y0, y1 = o0.krylov_vector(base, x), o1.krylov_vector(base, x)
    d = np.abs(y1 - y0).max() / np.abs(y0).max()
    assert 0 < d < 1e-6, d
    rng = np.random.default_rng(4)
    b = rng.standard_normal(n[::-1])
    b -= b.mean()
    p0, p1 = o0.poisson(b), o1.poisson(b)
    assert np.abs(p1 - p0).max() < 1e-6 * np.abs(p0).max()


# --- Section 3.1's special cases on the stretched grid ----------------------------------------------
def test_stretched_conduction_spectrum_is_kronecker_sum():
    """U = 0, Theta = 0: the temperature block is kappa times the Laplacian with homogeneous
    Dirichlet walls (CC), a sum of 1D operators along the three axes, so its eigenvalues are the
    sums of the 1D eigenvalues (the structure of Eq 17), here for the stretched 1D operators."""
    n = (4, 5, 3)
    nx, ny, nz = n
    gr, pr = 1.0e6, 0.71
    kappa = 1 / (pr * gr ** 0.5)
    o = Oracle(*n, gr=gr, pr=pr, stretch=S)
    base = np.zeros((4,) + o.shape)
    cols = []
    for k in range(1, nz + 1):
        for j in range(1, ny + 1):
            for i in range(1, nx + 1):
                x = np.zeros((4,) + o.shape)
                x[3, k, j, i] = 1.0
                cols.append(o.krylov_vector(base, x)[3, 1:-1, 1:-1, 1:-1].ravel())
    ev = np.sort(np.linalg.eigvals(np.array(cols).T).real)

    def dirichlet_1d(m):
        c, dx = positions(m, False, S), cell_widths(m, S)  # c[0] = 0 and c[m + 1] = 1 are the walls
        M = np.zeros((m, m))
        for t in range(1, m + 1):
            wl, wr = 1 / ((c[t] - c[t - 1]) * dx[t - 1]), 1 / ((c[t + 1] - c[t]) * dx[t - 1])
            M[t - 1, t - 1] = -(wl + wr)
            if t > 1:
                M[t - 1, t - 2] = wl
            if t < m:
                M[t - 1, t] = wr
        return np.linalg.eigvals(M).real

    lx, ly, lz = dirichlet_1d(nx), dirichlet_1d(ny), dirichlet_1d(nz)
    expect = np.sort((kappa * (lz[:, None, None] + ly[None, :, None] + lx[None, None, :])).ravel())
    assert np.allclose(ev, expect, rtol=1e-10)


@pytest.mark.parametrize("bc", [synth.CC, synth.AA])
def test_stretched_finite_difference_of_residual_equals_krylov_vector(bc):
    """The residual of Eqs (1)-(2) is quadratic in the state, so its central difference equals
    the Krylov vector exactly (up to rounding) on the stretched grid too."""
    n = (6, 7, 5)
    o = Oracle(*n, bc=bc, gr=2.0e6, stretch=S)
    St = packed_base(*n, bc, 41)
    x = o.project_input(rand_vec(*n, 42))
    eps = 1e-3
    Fp, _ = o.newton_residual(St + eps * x)
    Fm, _ = o.newton_residual(St - eps * x)
    y = o.krylov_vector(St, x)
    assert np.linalg.norm((Fp - Fm) / (2 * eps) - y) < 1e-10 * np.linalg.norm(y)
