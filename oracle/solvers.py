"""Krylov solvers and the Newton iteration around the Krylov-vector map (test infrastructure
only: tests/, __graft_entry__.smoke() and bench.py's CPU legs may call this module; the product
path never does).

Section 2 of the paper states the Newton method (steps 1-4: residual F of the steady equations,
solve the Jacobian system J [u, p, theta] = F, update U -> U - u, ...), and Section 3.1 names
the linear solvers: GMRES restarted after every 100 Krylov vectors until it saturates, then
BiCGstab(2) started from GMRES's last approximation. The paper defers the solvers to its
reference [17]; they are restated here from their published definitions:

* GMRES(m): Saad and Schultz (1986). Arnoldi basis of the Krylov space of the residual, the
  small least-squares problem reduced to triangular form by Givens rotations, restarted.
* BiCGstab(l): Sleijpen and Fokkema (1993), with l = 2: l BiCG steps, then a minimal-residual
  polynomial of degree l over the l + 1 residuals (modified Gram-Schmidt form).

All arithmetic is numpy FP64 on flat vectors; `matvec` is any callable x -> A x (the oracle's
Krylov-vector map, or a dense matrix in the pins).
"""
from __future__ import annotations

import numpy as np


def _dot(a, b):
    return float(np.dot(a.ravel(), b.ravel()))


def _norm(a):
    return float(np.sqrt(_dot(a, a)))


def arnoldi_cgs2(matvec, V, j):
    """One Arnoldi step: w = A v_j orthogonalised against v_0..v_j by classical Gram-Schmidt
    applied twice; V[j + 1] = w / ||w||. Returns the Hessenberg column h[0..j+1]."""
    w = matvec(V[j])
    h = np.zeros(j + 2)
    for _ in range(2):
        c = np.array([_dot(V[i], w) for i in range(j + 1)])
        for i in range(j + 1):
            w = w - c[i] * V[i]
        h[: j + 1] += c
    h[j + 1] = _norm(w)
    V[j + 1] = w / h[j + 1] if h[j + 1] > 0 else 0.0 * w
    return h


def gmres(matvec, b, x0, m, max_restarts, tol, sat=0.99):
    """Restarted GMRES(m) for A x = b from x0.

    A cycle starts from r = b - A x, builds up to m Arnoldi vectors, keeps the residual norm of
    the least-squares iterate with Givens rotations, stops early once that norm is at most
    tol ||b||, and adds V y to x. Cycles repeat until the residual at the start of a cycle is at
    most tol ||b|| (converged), or is above sat times the previous cycle's (saturated: the
    paper's signal to hand over to BiCGstab(2)), or max_restarts cycles have run.

    Returns (x, info) with info: restarts, iterations (Arnoldi steps), matvecs, converged,
    saturated, rel_residual (||b - A x|| / ||b|| recomputed at exit), history (residual norm at
    each cycle start)."""
    x = np.array(x0, dtype=np.float64, copy=True)
    bnorm = _norm(b)
    info = dict(restarts=0, iterations=0, matvecs=0, converged=False, saturated=False, history=[])
    prev = None
    shape = b.shape
    for _ in range(max_restarts):
        r = b - matvec(x)
        info["matvecs"] += 1
        beta = _norm(r)
        info["history"].append(beta)
        if beta <= tol * bnorm:
            info["converged"] = True
            break
        if prev is not None and beta > sat * prev:
            info["saturated"] = True
            break
        prev = beta
        info["restarts"] += 1
        V = np.zeros((m + 1,) + shape)
        V[0] = r / beta
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        k = 0
        for j in range(m):
            H[: j + 2, j] = arnoldi_cgs2(matvec, V, j)
            info["matvecs"] += 1
            info["iterations"] += 1
            # earlier rotations on the new column, then the rotation that zeroes H[j+1, j]
            for i in range(j):
                a, c = H[i, j], H[i + 1, j]
                H[i, j], H[i + 1, j] = cs[i] * a + sn[i] * c, -sn[i] * a + cs[i] * c
            d = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = (1.0, 0.0) if d == 0.0 else (H[j, j] / d, H[j + 1, j] / d)
            H[j, j], H[j + 1, j] = d, 0.0
            g[j], g[j + 1] = cs[j] * g[j], -sn[j] * g[j]
            k = j + 1
            if abs(g[j + 1]) <= tol * bnorm:
                break
        # back substitution R y = g[0:k]
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
        for i in range(k):
            x = x + y[i] * V[i]
    r = b - matvec(x)
    info["matvecs"] += 1
    info["rel_residual"] = _norm(r) / bnorm if bnorm > 0 else 0.0
    if info["rel_residual"] <= tol:
        info["converged"] = True
    return x, info


def bicgstab2(matvec, b, x0, max_iter, tol):
    """BiCGstab(2) for A x = b from x0 (shadow residual r~0 = r0). One iteration = two BiCG
    steps (four products with A) and the degree-2 minimal-residual update. Stops when
    ||r|| <= tol ||b||, after max_iter iterations, or on a breakdown: a zero or non-finite
    denominator (rho, the BiCG step's <u, r~0>, or a minimal-residual sigma), where the
    iteration cannot continue; x is then the last complete iterate.

    Returns (x, info): iterations, matvecs, converged, breakdown, rel_residual (recomputed at
    exit), history (||r|| after each iteration)."""
    x = np.array(x0, dtype=np.float64, copy=True)
    bnorm = _norm(b)
    r0 = b - matvec(x)
    info = dict(iterations=0, matvecs=1, converged=False, breakdown=False, history=[])
    rt = r0.copy()                          # shadow residual
    rh = [r0, np.zeros_like(b), np.zeros_like(b)]   # r^_0 .. r^_2
    uh = [np.zeros_like(b), np.zeros_like(b), np.zeros_like(b)]  # u^_0 .. u^_2
    rho0, alpha, omega = 1.0, 0.0, 1.0
    if _norm(r0) <= tol * bnorm:
        info["converged"] = True
    def bad(d):
        return d == 0.0 or not np.isfinite(d)

    while not info["converged"] and info["iterations"] < max_iter:
        rho0 = -omega * rho0
        xs = x  # the last complete iterate (kept on a breakdown)
        # BiCG part: l = 2 steps
        for j in range(2):
            rho1 = _dot(rh[j], rt)
            if bad(rho0):
                info["breakdown"] = True
                break
            beta = alpha * rho1 / rho0
            rho0 = rho1
            for i in range(j + 1):
                uh[i] = rh[i] - beta * uh[i]
            uh[j + 1] = matvec(uh[j])
            gamma = _dot(uh[j + 1], rt)
            if bad(gamma):
                info["breakdown"] = True
                break
            alpha = rho0 / gamma
            for i in range(j + 1):
                rh[i] = rh[i] - alpha * uh[i + 1]
            rh[j + 1] = matvec(rh[j])
            x = x + alpha * uh[0]
            info["matvecs"] += 2
        if info["breakdown"]:
            x = xs
            break
        # MR part (modified Gram-Schmidt on r^_1, r^_2)
        sigma1 = _dot(rh[1], rh[1])
        if bad(sigma1):
            info["breakdown"] = True
            x = xs
            break
        g1p = _dot(rh[0], rh[1]) / sigma1
        tau12 = _dot(rh[2], rh[1]) / sigma1
        rh[2] = rh[2] - tau12 * rh[1]
        sigma2 = _dot(rh[2], rh[2])
        if bad(sigma2):
            info["breakdown"] = True
            x = xs
            break
        g2p = _dot(rh[0], rh[2]) / sigma2
        g2 = g2p
        omega = g2
        g1 = g1p - tau12 * g2
        g1pp = g2
        x = x + g1 * rh[0]
        rh[0] = rh[0] - g2p * rh[2]
        uh[0] = uh[0] - g2 * uh[2]
        uh[0] = uh[0] - g1 * uh[1]
        x = x + g1pp * rh[1]
        rh[0] = rh[0] - g1p * rh[1]
        info["iterations"] += 1
        rn = _norm(rh[0])
        info["history"].append(rn)
        if rn <= tol * bnorm:
            info["converged"] = True
    r = b - matvec(x)
    info["matvecs"] += 1
    info["rel_residual"] = _norm(r) / bnorm if bnorm > 0 else 0.0
    info["converged"] = info["rel_residual"] <= tol
    return x, info


def newton(oracle, S0, max_newton, tol, m, max_restarts, lin_tol, sat, bicg_max_iter):
    """The Newton method of Section 2 on the oracle's discretisation: F = the projected steady
    residual of S (oracle.newton_residual); stop once ||F|| < tol; solve A d = F, A the Krylov
    map at the base S, by GMRES(m) restarted until it converges or saturates, then BiCGstab(2)
    from GMRES's last approximation if it has not converged, keeping whichever correction has the
    smaller recomputed residual; S <- S - d. A BiCGstab(2) correction preferred that way is still
    dropped for GMRES's when the Newton step with it does not decrease ||F|| (a correction can
    have the smaller linear residual and still carry a large part the linear residual does not
    see, as once happened near convergence in mixed precision).

    Returns (S, info): iterations, matvecs, res_norms (||F|| at each Newton step start),
    converged, bicg_rejected (BiCGstab(2) results not taken)."""
    S = np.array(S0, dtype=np.float64, copy=True)
    info = dict(iterations=0, matvecs=0, res_norms=[], converged=False, bicg_rejected=0)
    for _ in range(max_newton + 1):
        F, nrm = oracle.newton_residual(S)
        info["res_norms"].append(nrm)
        if nrm < tol:
            info["converged"] = True
            break
        if info["iterations"] == max_newton:
            break

        def matvec(x, S=S):
            return oracle.krylov_vector(S, x)

        d, gi = gmres(matvec, F, np.zeros_like(F), m, max_restarts, lin_tol, sat)
        info["matvecs"] += gi["matvecs"]
        if not gi["converged"]:
            d2, bi = bicgstab2(matvec, F, d, bicg_max_iter, lin_tol)
            info["matvecs"] += bi["matvecs"]
            # BiCGstab(2) replaces GMRES's correction only with a smaller recomputed residual
            # (started at the rounding level of the Krylov vectors it can stagnate or diverge)
            if bi["rel_residual"] < gi["rel_residual"] and oracle.newton_residual(S - d2)[1] <= nrm:
                d = d2
            else:
                info["bicg_rejected"] += 1
        S = S - d
        info["iterations"] += 1
    return S, info


# ---- Chebyshev-preconditioned Arnoldi for the rightmost eigenvalues (Eq (10)) ----------------
#
# Section 3.1 computes the leading eigenvalues of the Jacobian by the Chebyshev-preconditioned
# Arnoldi iteration (the paper uses ARPACK or HSL's EB13). Restated from Saad's Arnoldi-Chebyshev
# method (Math. Comp. 42, 1984): m Arnoldi steps give Ritz values; the unwanted ones are
# enclosed in an ellipse centred on the real axis; the next starting vector is the wanted Ritz
# vectors' real and imaginary parts filtered by the Chebyshev polynomial T_k((A - d) / c) of that
# ellipse, normalised at the rightmost wanted Ritz value, which damps the unwanted part of the
# spectrum; repeat until the wanted Ritz pairs' residuals are small. The filtered vector is
# multiplied by A once more: the Krylov map is singular on the full packed vector (its input
# projection zeroes the wall entries, its output projection the gradient fields), and for a
# stable spectrum that eigenvalue 0 lies right of the wanted eigenvalues, where the filter
# amplifies; the product removes those rounding-level components.


def ritz_pairs(H):
    """Ritz values of the Arnoldi matrix H ((k+1) x k), sorted by decreasing real part, their
    coefficient vectors and the residual norms |h_{k+1,k}| |y_k| / ||y|| (Arnoldi relation)."""
    k = H.shape[1]
    theta, Y = np.linalg.eig(H[:k, :k])
    order = np.argsort(-theta.real, kind="stable")
    theta, Y = theta[order], Y[:, order]
    res = np.abs(H[k, k - 1]) * np.abs(Y[k - 1, :]) / np.linalg.norm(Y, axis=0)
    return theta, Y, res


def wanted_count(theta, nev):
    """nev, plus one when the nev-th Ritz value is complex and its conjugate comes next (a
    conjugate pair is kept together)."""
    n = min(nev, len(theta))
    if n < len(theta) and theta[n - 1].imag != 0.0 and abs(theta[n] - np.conj(theta[n - 1])) <= \
            1e-12 * max(abs(theta[n - 1]), 1e-300):
        n += 1
    return n


def enclosing_ellipse(points):
    """The ellipse centred on the real axis with axes along the coordinate axes that encloses the
    points: its centre d and the square of its focal distance c2 = a^2 - b^2 (a: real semi-axis,
    b: imaginary semi-axis; c2 < 0 for an ellipse taller than wide). Semi-axes start at half the
    real extent and the largest |imaginary part| and grow by a common factor until every point is
    inside."""
    re, im = points.real, np.abs(points.imag)
    d = 0.5 * (re.max() + re.min())
    span = max(re.max() - re.min(), im.max(), 1e-300)
    a = max(0.5 * (re.max() - re.min()), 1e-8 * span)
    b = max(im.max(), 1e-8 * span)
    s = max(1.0, float(np.max(((re - d) / a) ** 2 + (im / b) ** 2)))
    a, b = a * np.sqrt(s), b * np.sqrt(s)
    return d, a * a - b * b


def chebyshev_filter(matvec, v, k, d, c2, lam):
    """T_k((A - d) / c) v / T_k((lam - d) / c) for real d, lam (lam > d) and real c2 = c^2, by the
    three-term recurrence written with the real quantities tau_j = sigma_j / c, where
    sigma_1 = c / (lam - d) and sigma_{j+1} = 1 / (2 (lam - d) / c - sigma_j):
    y_1 = tau_1 (A - d) y_0, y_{j+1} = 2 tau_{j+1} (A - d) y_j - tau_j tau_{j+1} c2 y_{j-1}."""
    e = lam - d
    tau = 1.0 / e
    y_prev = v
    y = tau * (matvec(v) - d * v)
    for _ in range(1, k):
        tau_next = 1.0 / (2.0 * e - tau * c2)
        y_next = 2.0 * tau_next * (matvec(y) - d * y) - tau * tau_next * c2 * y_prev
        y_prev, y, tau = y, y_next, tau_next
    return y


def arnoldi_chebyshev(matvec, v0, m, nev, k, tol, max_cycles):
    """Rightmost eigenvalues of A: cycles of m Arnoldi steps (classical Gram-Schmidt twice), each
    restarted from the wanted Ritz vectors filtered by a degree-k Chebyshev polynomial.
    Converged when every wanted Ritz pair has residual <= tol |theta|. nev = 1 asks for the
    leading eigenvalue (with its conjugate when complex), the case Section 3.1 computes; for
    nev > 1 on a non-normal A the later wanted values can be spurious (no locking of converged
    Schur vectors here).

    A cycle stops early once the new subdiagonal entry of H is at most tol times its column's
    norm (after at least nev steps; at once when it is exactly 0): the Krylov space then holds an
    invariant subspace to within tol, whose Ritz values are the answer. Otherwise the Ritz values
    of the rest of the space, which for a non-normal A lie anywhere in its field of values, could
    pass for rightmost eigenvalues.

    Returns (theta, res, info): the wanted Ritz values and residuals of the cycle with the
    smallest largest relative residual; info: cycles, matvecs, converged, ellipses (d, c2)
    used."""
    info = dict(cycles=0, matvecs=0, converged=False, ellipses=[])
    v = np.array(v0, dtype=np.float64, copy=True)
    shape = v.shape
    theta = res = None
    best = (np.inf, None, None)  # the wanted set with the smallest largest relative residual
    for _ in range(max_cycles):
        info["cycles"] += 1
        V = np.zeros((m + 1,) + shape)
        V[0] = v / _norm(v)
        H = np.zeros((m + 1, m))
        kk = m
        for j in range(m):
            H[: j + 2, j] = arnoldi_cgs2(matvec, V, j)
            info["matvecs"] += 1
            # the space holds an invariant subspace to within tol (after at least nev steps), or
            # exactly: stop the cycle there
            hn, col = H[j + 1, j], np.linalg.norm(H[: j + 2, j])
            if hn == 0.0 or (hn <= tol * col and j + 1 >= nev):
                kk = j + 1
                break
        th, Y, rs = ritz_pairs(H[: kk + 1, :kk])
        nw = wanted_count(th, nev)
        theta, res = th[:nw], rs[:nw]
        score = float(np.max(res / np.maximum(np.abs(theta), 1e-300)))
        if score < best[0]:
            best = (score, theta, res)
        if score <= tol:
            info["converged"] = True
            break
        # restart vector: the wanted Ritz vectors' real and imaginary parts, each normalised
        coef = np.zeros(kk)
        for i in range(nw):
            y = Y[:, i] / np.linalg.norm(Y[:, i])
            coef += y.real + y.imag
        v = np.tensordot(coef, V[:kk], axes=1)
        # Chebyshev filter over the ellipse of the unwanted Ritz values
        if nw >= kk:
            continue
        d, c2 = enclosing_ellipse(th[nw:])
        lam = theta[0].real
        if lam > d:
            info["ellipses"].append((d, c2))
            v = chebyshev_filter(matvec, v, k, d, c2, lam)
            # one product with A: the Krylov map's null space (entries outside its range, where
            # the filter's polynomial is large when the spectrum is stable) holds rounding-level
            # components of the filtered vector; A removes them
            v = matvec(v)
            info["matvecs"] += k + 1
    # once the wanted eigenvector has converged as far as rounding allows, the next Krylov
    # directions are rounding noise and later cycles can rank a spurious Ritz value first:
    # return the best wanted set seen
    if best[1] is not None:
        theta, res = best[1], best[2]
    return theta, res, info
