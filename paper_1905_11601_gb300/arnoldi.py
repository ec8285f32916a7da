"""Arnoldi driver for the eigenvalue problem Eq (10) over the GPU Krylov map.

The basis and every Krylov vector live on the GPU (kv_arnoldi_step); only the small Hessenberg
matrix H comes back to the host, where its eigenvalues (the Ritz values) are computed. The
residual of a Ritz pair (theta, X = V y) follows from the Arnoldi relation A V_k = V_k H_k +
h_{k+1,k} v_{k+1} e_k^T as |h_{k+1,k}| |y_k| / ||y||, the quantity the paper monitors
(||J X - lambda X|| / ||X||, Section 3.1).
"""
from __future__ import annotations

import numpy as np


def arnoldi(grid, v0, k):
    """k Arnoldi steps from v0 (a packed vector, device): returns V ((k+1) x packed) and H."""
    torch = grid.torch
    V = torch.zeros((k + 1, 4) + grid.shape, dtype=torch.float64, device="cuda")
    V[0] = v0 / torch.linalg.vector_norm(v0)
    H = np.zeros((k + 1, k))
    for j in range(k):
        H[: j + 2, j] = grid.arnoldi_step(V, j)
    return V, H


def ritz(H, nev):
    """The nev Ritz values with the largest real parts, their coefficient vectors y (columns)
    and the Arnoldi residual estimates |h_{k+1,k}| |y_k| / ||y||."""
    k = H.shape[1]
    theta, Y = np.linalg.eig(H[:k, :k])
    order = np.argsort(-theta.real)[:nev]
    theta, Y = theta[order], Y[:, order]
    res = np.abs(H[k, k - 1]) * np.abs(Y[k - 1, :]) / np.linalg.norm(Y, axis=0)
    return theta, Y, res


def ritz_vector(V, y):
    """X = V_k y (complex coefficients give a complex vector as a (real, imag) pair)."""
    import torch

    k = y.shape[0]
    Vk = V[:k].reshape(k, -1)
    yr = torch.from_numpy(np.ascontiguousarray(y.real)).to(Vk)
    yi = torch.from_numpy(np.ascontiguousarray(y.imag)).to(Vk)
    return (yr @ Vk).reshape(V.shape[1:]), (yi @ Vk).reshape(V.shape[1:])


def save_state(path, V, H, j):
    """Checkpoint of an Arnoldi run: the basis V (moved to host memory), H and the step count."""
    import torch

    torch.save({"V": V.detach().cpu(), "H": np.asarray(H), "j": int(j)}, path)


def load_state(path, device="cuda"):
    """Restores (V, H, j) saved by save_state; V is placed on `device`."""
    import torch

    d = torch.load(path, weights_only=False)
    return d["V"].to(device), np.asarray(d["H"]), int(d["j"])
