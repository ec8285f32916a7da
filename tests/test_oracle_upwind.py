"""Pins of the oracle's optional first-order upwind advection (adv = 1), CPU only.

The paper's discretisation (Eqs (8)-(9), Section 3) is the central one; upwinding is an option
of the library. Its reading: along each axis the derivative of an advected field is the
one-sided difference towards the upstream neighbour, picked by the sign of the base velocity
averaged to the node (>= 0: backward), over the actual node gap. The linearised operator keeps
the base velocity's choice in both advection terms. These tests check that reading against an
independent Kronecker assembly, a textbook special case, finite differences of the upwind
residual, and the definition of the transpose.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_1905_11601_gb300 import synth
from tests.mac_assembly import MacOps

UP = 1


def packed_base(nx, ny, nz, bc, seed):
    return np.stack(synth.base_flow(nx, ny, nz, bc, seed))


def rand_vec(nx, ny, nz, seed):
    return synth.krylov_input(nx, ny, nz, seed)[0]


@pytest.mark.parametrize("n,bc,s", [((4, 4, 4), synth.CC, 0.0), ((5, 4, 6), synth.CC, 0.0),
                                    ((5, 4, 6), synth.AA, 0.0), ((6, 5, 7), synth.AA, 0.1)])
def test_upwind_jacobian_matches_kronecker_assembly(n, bc, s):
    o = Oracle(*n, bc=bc, gr=2.0e6, pr=0.71, stretch=s, adv=UP)
    base = packed_base(*n, bc, 21)
    xp = o.project_input(rand_vec(*n, 22))
    J = MacOps(*n, s=s).jacobian(base, 2.0e6, 0.71, upwind=True)
    y_asm = (J @ xp.ravel()).reshape(xp.shape)
    y_or = o.jx_raw(base, xp)
    assert np.allclose(y_or, y_asm, rtol=0, atol=1e-12 * np.abs(y_asm).max())
    # and it is not the central operator (the base flow has both signs on every axis)
    y_c = Oracle(*n, bc=bc, gr=2.0e6, pr=0.71, stretch=s).jx_raw(base, xp)
    assert np.abs(y_c - y_or).max() > 1e-3 * np.abs(y_or).max()


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_uniform_velocity_gives_one_sided_differences(sign):
    """A constant base velocity c (every velocity entry, no temperature gradient): away from the
    walls the advection terms of J x reduce to -c times the backward (c > 0) or forward (c < 0)
    difference of each field, and the gradient terms of the base vanish."""
    n = (7, 6, 8)
    gr, pr = 1.0e6, 0.71
    nu, kappa = gr ** -0.5, 1.0 / (pr * gr ** 0.5)
    c0 = 0.37 * sign
    base = np.zeros((4,) + synth.padded_shape(*n))
    base[:3] = c0
    x = rand_vec(*n, 5)
    y = Oracle(*n, gr=gr, pr=pr, adv=UP).jx_raw(base, x)
    nx, ny, nz = n
    inv = (nx, ny, nz)  # 1/h per axis: x (last index), y, z (first)
    for F in range(4):
        f = x[F]
        sl = (slice(2, -2),) * 3

        def shift(a, d):  # value at index + d along axis a (0 = x)
            ax = 2 - a
            return np.roll(f, -d, axis=ax)

        lap = sum((shift(a, 1) - 2 * f + shift(a, -1)) * inv[a] ** 2 for a in range(3))
        if sign > 0:
            adv = sum((f - shift(a, -1)) * inv[a] for a in range(3))
        else:
            adv = sum((shift(a, 1) - f) * inv[a] for a in range(3))
        expect = (kappa if F == 3 else nu) * lap - c0 * adv
        if F == 2:
            expect = expect + 0.5 * (x[3] + np.roll(x[3], -1, axis=0))
        assert np.allclose(y[F][sl], expect[sl], rtol=0, atol=1e-12 * np.abs(expect[sl]).max()), F


def test_upwind_matches_central_for_linear_fields_in_the_interior():
    """One-sided and central differences of a linear field agree (both exact)."""
    n = (8, 7, 9)
    rng = np.random.default_rng(5)

    def coords(F):
        xs = [synth.face_coords(n[0]) if F == 0 else synth.cell_coords(n[0]),
              synth.face_coords(n[1]) if F == 1 else synth.cell_coords(n[1]),
              synth.face_coords(n[2]) if F == 2 else synth.cell_coords(n[2])]
        Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
        return Z, Y, X

    def lin(c, Z, Y, X):
        return c[0] + c[1] * X + c[2] * Y + c[3] * Z

    cb, cx = rng.standard_normal((4, 4)), rng.standard_normal((4, 4))
    base = np.stack([lin(cb[F], *coords(F)) for F in range(4)])
    x = np.stack([lin(cx[F], *coords(F)) for F in range(4)])
    yu = Oracle(*n, adv=UP).jx_raw(base, x)
    yc = Oracle(*n).jx_raw(base, x)
    sl = (slice(2, -2),) * 3
    for F in range(4):
        assert np.allclose(yu[F][sl], yc[F][sl], rtol=0, atol=1e-11 * np.abs(yc[F][sl]).max()), F


def _selector_margin(n, S, x):
    """The largest eps for which no averaged velocity of S + t x (|t| <= eps) changes sign at a
    node where an equation is formed, with a factor 10 to spare."""
    ops = MacOps(*n)
    worst = np.inf
    for F in range(4):
        m = ops.dof_mask(F) > 0
        for c in range(3):
            a = (ops.interp(c, F) @ S[c].ravel())[m]
            da = np.abs(ops.interp(c, F) @ x[c].ravel())[m]
            k = da > 0
            worst = min(worst, np.min(np.abs(a[k]) / da[k]))
    return 0.1 * worst


@pytest.mark.parametrize("bc", [synth.CC, synth.AA])
def test_finite_difference_of_upwind_residual_equals_krylov_vector(bc):
    """With the one-sided choices fixed, the upwind residual is quadratic in the state, so its
    central difference is the linearised operator exactly (to rounding) when eps is small
    enough that no choice changes between S - eps x and S + eps x."""
    n = (6, 7, 5)
    o = Oracle(*n, bc=bc, gr=2.0e6, adv=UP)
    S = packed_base(*n, bc, 41)
    x = o.project_input(rand_vec(*n, 42))
    eps = min(1e-3, _selector_margin(n, S, x))
    assert eps > 1e-9, eps
    Fp, _ = o.newton_residual(S + eps * x)
    Fm, _ = o.newton_residual(S - eps * x)
    fd = (Fp - Fm) / (2 * eps)
    y = o.krylov_vector(S, x)
    assert np.linalg.norm(fd - y) < max(1e-10, 1e-15 / eps) * np.linalg.norm(y)
    # the central operator is not what the upwind residual linearises to
    yc = Oracle(*n, bc=bc, gr=2.0e6).krylov_vector(S, x)
    assert np.linalg.norm(yc - y) > 1e-3 * np.linalg.norm(y)


@pytest.mark.parametrize("n,bc", [((6, 5, 7), synth.CC), ((5, 6, 4), synth.AA)])
def test_upwind_adjoint_dot_product(n, bc):
    o = Oracle(*n, bc=bc, gr=2e6, adv=UP)
    base = packed_base(*n, bc, 71)
    x = synth.krylov_input(*n, 72, 2)
    xp = o.project_input(x[0])
    lhs, rhs = np.vdot(x[1], o.jx_raw(base, xp)), np.vdot(o.jt_raw(base, x[1]), xp)
    assert abs(lhs - rhs) < 1e-13 * np.linalg.norm(x[1]) * np.linalg.norm(o.jx_raw(base, xp))
    A = o.krylov_vector(base, x[0])
    lhs, rhs = np.vdot(x[1], A), np.vdot(o.krylov_adjoint(base, x[1]), x[0])
    assert abs(lhs - rhs) < 1e-13 * np.linalg.norm(x[1]) * np.linalg.norm(A)


def test_upwind_jt_matches_transpose_of_kronecker_assembly():
    n = (5, 4, 6)
    o = Oracle(*n, gr=2e6, adv=UP)
    base = packed_base(*n, synth.CC, 73)
    ys = rand_vec(*n, 74)
    J = MacOps(*n).jacobian(base, 2e6, 0.71, upwind=True)
    z_asm = (J.T @ ys.ravel()).reshape(ys.shape)
    assert np.allclose(o.jt_raw(base, ys), z_asm, rtol=0, atol=1e-12 * np.abs(z_asm).max())


def test_base_gradient_is_not_defined_for_upwind():
    n = (4, 4, 4)
    o = Oracle(*n, adv=UP)
    x = rand_vec(*n, 3)
    assert np.isnan(o.grad_base(o.project_input(x), x)).all()


def test_invalid_scheme_is_refused():
    with pytest.raises(ValueError):
        Oracle(4, 4, 4, adv=2)
