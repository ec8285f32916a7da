"""Seeded synthetic inputs for the Krylov-vector path of a laterally heated cube.

This module is shared by the tests, the benchmark and the CPU oracle's callers. It holds
no arithmetic of the method itself (no Jacobian, no Poisson solve, no projection): it only
draws seeded random numbers and evaluates the closed-form base-flow recipe on the grid.

Grid convention (a MAC / staggered finite-volume grid of the unit cube, uniform spacing
h_a = 1/n_a per axis; Section 3.1 discretises Eqs (1)-(7) on such a grid):

* every field is stored as a padded array of shape (nz+2, ny+2, nx+2), x fastest;
* along an axis a "cell-like" index i = 1..n sits at (i - 1/2) h and indices 0 and n+1 are
  wall nodes lying on the walls (coordinates 0 and 1);
* a "face-like" index i = 0..n sits at i h (index n+1 is unused padding);
* T and p are cell-like on all axes; u is face-like along x, v along y, w along z.

The base flow stands in for the converged steady states of Section 4 (which are not
available): Theta = 1 - x + 0.05 * (sum of 8 seeded sine-mode products that vanish on the
walls), with the wall values of Eqs (4)-(7); the velocity is the discrete curl of a seeded
edge-located vector potential with sin^2 wall factors, so its discrete divergence is zero to
rounding and it is no-slip, scaled to max |U| = 0.1.
"""
from __future__ import annotations

import dataclasses
import numpy as np

CC = 0  # conducting spanwise walls, Eq (6)
AA = 1  # insulated spanwise walls, Eq (7)


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic workload: grid, parameters and seed."""

    name: str
    nx: int
    ny: int
    nz: int
    bc: int
    gr: float
    pr: float
    seed: int


# The workloads: a small parity case, the plain FP64 Arnoldi grid, the mixed-precision grid
# with insulated spanwise walls, the adjoint grid and the 256^3 grid of the throughput metric.
WORKLOADS = {
    "cube16_cc": Workload("cube16_cc", 16, 16, 16, CC, 1.0e6, 0.71, 11601 + 0),
    "cube100_cc": Workload("cube100_cc", 100, 100, 100, CC, 2.0e6, 0.71, 11601 + 1),
    "cube128_aa": Workload("cube128_aa", 128, 128, 128, AA, 3.0e6, 0.71, 11601 + 2),
    "cube160_cc": Workload("cube160_cc", 160, 160, 160, CC, 2.5e6, 0.71, 11601 + 3),
    "cube256_cc": Workload("cube256_cc", 256, 256, 256, CC, 3.3429e6, 0.71, 11601 + 4),
}


def padded_shape(nx: int, ny: int, nz: int) -> tuple[int, int, int]:
    return (nz + 2, ny + 2, nx + 2)


def cell_coords(n: int) -> np.ndarray:
    """Coordinates of cell-like indices 0..n+1 (wall nodes on the walls)."""
    c = (np.arange(n + 2, dtype=np.float64) - 0.5) / n
    c[0] = 0.0
    c[n + 1] = 1.0
    return c


def face_coords(n: int) -> np.ndarray:
    """Coordinates of face-like indices 0..n (index n+1 is padding, given coordinate 1)."""
    f = np.arange(n + 2, dtype=np.float64) / n
    f[n + 1] = 1.0
    return f


def _grid(xs, ys, zs):
    return np.meshgrid(zs, ys, xs, indexing="ij")  # arrays indexed [k, j, i]


def base_temperature(nx, ny, nz, bc, rng) -> np.ndarray:
    """Theta = 1 - x + 0.05 * sum_m a_m sin(p_m pi x) s(q_m pi y) sin(r_m pi z), wall values set."""
    a = rng.uniform(-1.0, 1.0, size=8)
    p = rng.integers(1, 5, size=8)
    q = rng.integers(1, 5, size=8)
    r = rng.integers(1, 5, size=8)
    xc, yc, zc = cell_coords(nx), cell_coords(ny), cell_coords(nz)
    th = np.broadcast_to(1.0 - xc[None, None, :], padded_shape(nx, ny, nz)).copy()
    for m in range(8):  # separable products, evaluated as outer products of 1D factors
        sx = np.sin(p[m] * np.pi * xc)
        sy = np.sin(q[m] * np.pi * yc) if bc == CC else np.cos(q[m] * np.pi * yc)
        sz = np.sin(r[m] * np.pi * zc)
        th += (0.05 * a[m]) * sz[:, None, None] * sy[None, :, None] * sx[None, None, :]
    # wall values: Eq (4) on x walls, Eq (5) on z walls, Eq (6) (CC) or a discrete Eq (7) (AA)
    th[:, :, 0] = 1.0
    th[:, :, nx + 1] = 0.0
    lin = 1.0 - xc[None, :]
    th[0, :, :] = lin
    th[nz + 1, :, :] = lin
    if bc == CC:
        th[:, 0, :] = lin
        th[:, ny + 1, :] = lin
    else:
        th[:, 0, :] = th[:, 1, :]
        th[:, ny + 1, :] = th[:, ny, :]
        th[:, :, 0] = 1.0
        th[:, :, nx + 1] = 0.0
        th[0, :, :] = lin
        th[nz + 1, :, :] = lin
    return th


def base_velocity(nx, ny, nz, rng, umax=0.1):
    """Discrete curl of an edge-located potential A = s(x)s(y)s(z) sum_m c_m cos(a pi x + b pi y + g pi z).

    s(t) = sin^2(pi t). A_x lives on x-edges (cell x, face y, face z), A_y on y-edges and A_z on
    z-edges. The discrete curl makes the discrete divergence vanish identically; every
    velocity entry outside the interior faces (wall-normal faces, tangential wall nodes,
    padding) is zero (no-slip).
    """
    xc, yc, zc = cell_coords(nx), cell_coords(ny), cell_coords(nz)
    xf, yf, zf = face_coords(nx), face_coords(ny), face_coords(nz)
    coef = rng.standard_normal(size=(3, 4))
    freq = rng.integers(0, 3, size=(3, 4, 3))

    def potential(comp, xs, ys, zs):
        # s(x)s(y)s(z) * sum_m c_m Re(exp(i a pi x) exp(i b pi y) exp(i g pi z)): separable
        acc = np.zeros((len(zs), len(ys), len(xs)))
        for m in range(4):
            al, be, ga = freq[comp, m]
            ex, ey, ez = np.exp(1j * al * np.pi * xs), np.exp(1j * be * np.pi * ys), np.exp(1j * ga * np.pi * zs)
            acc += coef[comp, m] * (ez[:, None, None] * ey[None, :, None] * ex[None, None, :]).real
        sx, sy, sz = np.sin(np.pi * xs) ** 2, np.sin(np.pi * ys) ** 2, np.sin(np.pi * zs) ** 2
        return acc * (sz[:, None, None] * sy[None, :, None] * sx[None, None, :])

    Ax = potential(0, xc, yf, zf)  # [k face, j face, i cell]
    Ay = potential(1, xf, yc, zf)  # [k face, j cell, i face]
    Az = potential(2, xf, yf, zc)  # [k cell, j face, i face]
    hx, hy, hz = 1.0 / nx, 1.0 / ny, 1.0 / nz
    shape = padded_shape(nx, ny, nz)
    U = np.zeros(shape)
    V = np.zeros(shape)
    W = np.zeros(shape)
    # u on x-faces i = 1..nx-1, cells j, k = 1..n
    i, j, k = slice(1, nx), slice(1, ny + 1), slice(1, nz + 1)
    U[k, j, i] = (Az[k, 1:ny + 1, i] - Az[k, 0:ny, i]) / hy - (Ay[1:nz + 1, j, i] - Ay[0:nz, j, i]) / hz
    i, j, k = slice(1, nx + 1), slice(1, ny), slice(1, nz + 1)
    V[k, j, i] = (Ax[1:nz + 1, j, i] - Ax[0:nz, j, i]) / hz - (Az[k, j, 1:nx + 1] - Az[k, j, 0:nx]) / hx
    i, j, k = slice(1, nx + 1), slice(1, ny + 1), slice(1, nz)
    W[k, j, i] = (Ay[k, j, 1:nx + 1] - Ay[k, j, 0:nx]) / hx - (Ax[k, 1:ny + 1, i] - Ax[k, 0:ny, i]) / hy
    scale = umax / max(np.abs(U).max(), np.abs(V).max(), np.abs(W).max(), 1e-300)
    return U * scale, V * scale, W * scale


def base_flow(nx, ny, nz, bc, seed):
    """(U, V, W, Theta) padded FP64 arrays for the given grid, spanwise BC and seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    th = base_temperature(nx, ny, nz, bc, rng)
    U, V, W = base_velocity(nx, ny, nz, rng)
    return U, V, W, th


def krylov_input(nx, ny, nz, seed, count=1):
    """`count` packed vectors (u | v | w | T), i.i.d. N(0, 1) on every stored entry.

    Returns an array of shape (count, 4, nz+2, ny+2, nx+2).
    """
    rng = np.random.Generator(np.random.PCG64([seed, 7]))
    return rng.standard_normal(size=(count, 4) + padded_shape(nx, ny, nz))


def workload_arrays(w: Workload, count=1):
    U, V, W, th = base_flow(w.nx, w.ny, w.nz, w.bc, w.seed)
    x = krylov_input(w.nx, w.ny, w.nz, w.seed, count)
    return (U, V, W, th), x
