"""Small compositions of oracle calls shared by the CPU pins and the GPU parity tests."""
import numpy as np


def velocity_masks(shape, n):
    nx, ny, nz = n
    m = [np.zeros(shape) for _ in range(3)]
    m[0][1:nz + 1, 1:ny + 1, 1:nx] = 1
    m[1][1:nz + 1, 1:ny, 1:nx + 1] = 1
    m[2][1:nz, 1:ny + 1, 1:nx + 1] = 1
    return np.stack(m)


def project_output_side(o, y):
    """(Pi_v (+) P_T) y with the oracle's pieces: mask, SIMPLE projection, Eq (21)."""
    vel = y[:3] * velocity_masks(o.shape, (o.nx, o.ny, o.nz))
    vel, _ = o.correct(o.poisson(o.divergence(vel)), vel)
    return np.concatenate([vel, o.tproj_gram(y[3])[None]])
