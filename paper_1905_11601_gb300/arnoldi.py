"""Arnoldi driver for the eigenvalue problem Eq (10) over the GPU Krylov map.

The basis and every Krylov vector live on the GPU (kv_arnoldi_run); only the small Hessenberg
matrix H comes back to the host, where its eigenvalues (the Ritz values) are computed. The
residual of a Ritz pair (theta, X = V y) follows from the Arnoldi relation A V_k = V_k H_k +
h_{k+1,k} v_{k+1} e_k^T as |h_{k+1,k}| |y_k| / ||y||, the quantity the paper monitors
(||J X - lambda X|| / ||X||, Section 3.1).
"""
from __future__ import annotations

import numpy as np

from .kv import KvError


def arnoldi(grid, v0, k):
    """k Arnoldi steps from v0 (a packed vector, device): returns V ((k+1) x packed) and H."""
    torch = grid.torch
    V = torch.zeros((k + 1, 4) + grid.shape, dtype=torch.float64, device="cuda")
    V[0] = v0 / torch.linalg.vector_norm(v0)
    H = np.zeros((k + 1, k))
    H[:, :] = grid.arnoldi_run(V, 0, k)  # one call: the delayed classical Gram-Schmidt
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


def _ellipse(points):
    """Centre d and squared focal distance c2 of the axis-aligned ellipse centred on the real
    axis that encloses the points (semi-axes from the points' real extent and largest |imag|,
    grown by a common factor until all are inside)."""
    re, im = points.real, np.abs(points.imag)
    d = 0.5 * (re.max() + re.min())
    span = max(re.max() - re.min(), im.max(), 1e-300)
    a = max(0.5 * (re.max() - re.min()), 1e-8 * span)
    b = max(im.max(), 1e-8 * span)
    s = max(1.0, float(np.max(((re - d) / a) ** 2 + (im / b) ** 2)))
    return d, s * (a * a - b * b)


def _wanted(theta, nev):
    n = min(nev, len(theta))
    if n < len(theta) and theta[n - 1].imag != 0.0 and \
            abs(theta[n] - np.conj(theta[n - 1])) <= 1e-12 * max(abs(theta[n - 1]), 1e-300):
        n += 1
    return n


def arnoldi_chebyshev(grid, v0, m=30, nev=1, k=20, tol=1e-10, max_cycles=100):
    """The leading eigenvalue(s) of Eq (10) by the Chebyshev-preconditioned Arnoldi iteration
    (Section 3.1; Saad's Arnoldi-Chebyshev method): cycles of m Arnoldi steps (kv_arnoldi_run);
    the unwanted Ritz values define an ellipse centred on the real axis; the wanted Ritz vectors'
    real and imaginary parts (kv_combine) are filtered by the degree-k Chebyshev polynomial of
    that ellipse, normalised at the rightmost wanted Ritz value (three-term recurrence over
    kv_krylov_vector and kv_axpby, real also for imaginary focal distances), multiplied by A once
    more (the Krylov map's null space, where the filter amplifies when the spectrum is stable,
    holds rounding-level components), and start the next cycle. A cycle stops once the new
    subdiagonal entry of H is at most tol times its column (after at least nev steps, or at
    once when exactly 0). Converged when every wanted Ritz pair has residual <= tol |theta|.
    nev = 1: the leading eigenvalue, with its conjugate when complex.

    v0: packed vector (device). Returns (theta, res, info) with the wanted Ritz values and their
    residuals from the cycle with the smallest largest relative residual, and info: cycles,
    matvecs, converged, ellipses, V (the last basis) and Y (the wanted Ritz coefficient vectors in
    it when the last cycle converged, else None)."""
    torch = grid.torch
    shape = (4,) + grid.shape
    V = torch.zeros((m + 1,) + shape, dtype=torch.float64, device="cuda")
    v, y_prev, y, w = (torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(4))
    info = dict(cycles=0, matvecs=0, converged=False, ellipses=[])
    grid.axpby(1.0, v0, 0.0, v)
    theta = res = Yw = None
    best = (np.inf, None, None, None)  # the wanted set with the smallest largest relative residual
    for _ in range(max_cycles):
        info["cycles"] += 1
        nv = np.sqrt(grid.dot(v, v))
        grid.axpby(1.0 / nv, v, 0.0, V[0])
        # the cycle's m steps as one kv_arnoldi_run (one synchronisation), cut at the first step
        # whose new vector is negligible; a breakdown inside the run (an invariant subspace)
        # repeats the cycle step by step, stopping there
        try:
            H = grid.arnoldi_run(V, 0, m)
            info["matvecs"] += m
        except KvError:
            H = None
        kk = m
        if H is not None:
            for j in range(m):
                hn, col = H[j + 1, j], np.linalg.norm(H[: j + 2, j])
                if hn == 0.0 or (hn <= tol * col and j + 1 >= nev):
                    kk = j + 1
                    break
        else:
            H = np.zeros((m + 1, m))
            for j in range(m):
                H[: j + 2, j] = grid.arnoldi_step(V, j)
                info["matvecs"] += 1
                hn, col = H[j + 1, j], np.linalg.norm(H[: j + 2, j])
                if hn == 0.0 or (hn <= tol * col and j + 1 >= nev):
                    kk = j + 1
                    break
        theta_all, Y, rs = ritz(H[: kk + 1, :kk], kk)
        nw = _wanted(theta_all, nev)
        theta, res, Yw = theta_all[:nw], rs[:nw], Y[:, :nw]
        score = float(np.max(res / np.maximum(np.abs(theta), 1e-300)))
        if score < best[0]:
            best = (score, theta, res, Yw)
        if score <= tol:
            info["converged"] = True
            break
        coef = np.zeros(kk)
        for i in range(nw):
            yi = Y[:, i] / np.linalg.norm(Y[:, i])
            coef += yi.real + yi.imag
        grid.combine(V, coef, v)
        if nw >= kk:
            continue
        d, c2 = _ellipse(theta_all[nw:])
        lam = theta[0].real
        if lam <= d:
            continue
        info["ellipses"].append((d, c2))
        # y_1 = tau_1 (A - d) v; y_{j+1} = 2 tau_{j+1} (A - d) y_j - tau_j tau_{j+1} c2 y_{j-1}
        e = lam - d
        tau = 1.0 / e
        grid.axpby(1.0, v, 0.0, y_prev)
        grid.krylov_vector(v, w)
        grid.axpby(-d, v, 1.0, w)
        grid.axpby(tau, w, 0.0, y)
        for _ in range(1, k):
            tau_next = 1.0 / (2.0 * e - tau * c2)
            grid.krylov_vector(y, w)
            grid.axpby(-d, y, 1.0, w)
            grid.axpby(-tau * tau_next * c2, y_prev, 2.0 * tau_next, w)
            y_prev, y, w = y, w, y_prev
            tau = tau_next
        grid.krylov_vector(y, v)  # the product that removes the null-space components
        info["matvecs"] += k + 1
    # the best wanted set seen (after the eigenvector has converged as far as rounding allows, the
    # next Krylov directions are noise and a later cycle can rank a spurious Ritz value first)
    converged_now = info["converged"]
    if best[1] is not None:
        theta, res = best[1], best[2]
        if not converged_now:
            Yw = None  # the best set's basis was overwritten by later cycles
    info["V"], info["Y"] = V, Yw
    return theta, res, info
