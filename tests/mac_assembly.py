"""Independent sparse assembly of the discrete operators, used only to pin the oracle.

The oracle applies its stencils point by point; this module builds the same operators as
sparse matrices from 1D factors combined with Kronecker products (the structure of Eq (14)).
A mistake in either (a wrong index, sign, spacing or interpolation weight) makes them differ.
Padded layout (nz+2, ny+2, nx+2), x fastest, so a 3D operator is kron(Mz, My, Mx).
A stretched grid (Eq 22, parameter s) maps the faces xi -> xi - s sin(2 pi xi); cell centres
are the midpoints of their faces, and each row of the flux-form Laplacian, the divergence and
the gradient divides by the width it spans (control volume, cell, centre gap).
"""
import numpy as np
import scipy.sparse as sp


def stretched_faces(n, s):
    """Face coordinates 0..n of Eq (22)."""
    xi = np.arange(n + 1) / n
    f = xi - s * np.sin(2 * np.pi * xi)
    f[0], f[n] = 0.0, 1.0
    return f


def positions(n, face, s=0.0):
    """Node coordinates of indices 0..n+1 along one axis."""
    if s != 0.0:
        f = stretched_faces(n, s)
        if face:
            return np.append(f, 2.0 - f[n - 1])  # padding, never used by an interior row
        p = np.empty(n + 2)
        p[0], p[n + 1] = 0.0, 1.0
        p[1:n + 1] = 0.5 * (f[:-1] + f[1:])
        return p
    if face:
        p = np.arange(n + 2) / n
        p[n + 1] = 1.0 + 1.0 / n  # padding, never used by an interior row
        return p
    p = (np.arange(n + 2) - 0.5) / n
    p[0], p[n + 1] = 0.0, 1.0
    return p


def interior_rows(n, face):
    return np.arange(1, n) if face else np.arange(1, n + 1)


def control_volume(n, face, s=0.0):
    """Width of the control volume of each node 0..n+1 (interior rows only are meaningful)."""
    if s == 0.0:
        return np.full(n + 2, 1.0 / n)
    w = np.ones(n + 2)
    if face:
        c = positions(n, False, s)
        w[1:n] = c[2:n + 1] - c[1:n]
    else:
        f = stretched_faces(n, s)
        w[1:n + 1] = f[1:] - f[:-1]
    return w


def d2_1d(n, face, s=0.0):
    p, h = positions(n, face, s), control_volume(n, face, s)
    M = sp.lil_matrix((n + 2, n + 2))
    for t in interior_rows(n, face):
        wl, wr = 1.0 / (p[t] - p[t - 1]), 1.0 / (p[t + 1] - p[t])
        M[t, t - 1] += wl / h[t]
        M[t, t + 1] += wr / h[t]
        M[t, t] -= (wl + wr) / h[t]
    return M.tocsr()


def d1_1d(n, face, s=0.0):
    p = positions(n, face, s)
    M = sp.lil_matrix((n + 2, n + 2))
    for t in interior_rows(n, face):
        dm, dp = p[t] - p[t - 1], p[t + 1] - p[t]
        den = dm * dp * (dm + dp)
        M[t, t + 1] += dm * dm / den
        M[t, t - 1] -= dp * dp / den
        M[t, t] += (dp * dp - dm * dm) / den
    return M.tocsr()


def d1_side_1d(n, face, backward, s=0.0):
    """One-sided first difference over the node gap: towards t-1 (backward) or t+1 (forward)."""
    p = positions(n, face, s)
    M = sp.lil_matrix((n + 2, n + 2))
    for t in interior_rows(n, face):
        if backward:
            g = p[t] - p[t - 1]
            M[t, t] += 1.0 / g
            M[t, t - 1] -= 1.0 / g
        else:
            g = p[t + 1] - p[t]
            M[t, t + 1] += 1.0 / g
            M[t, t] -= 1.0 / g
    return M.tocsr()


def face_to_cell(n):
    """Row t (cell-like node) = mean of faces t-1 and t."""
    M = sp.lil_matrix((n + 2, n + 2))
    for t in range(1, n + 1):
        M[t, t - 1] = 0.5
        M[t, t] = 0.5
    return M.tocsr()


def cell_to_face(n):
    """Row t (face node) = mean of cell-like nodes t and t+1."""
    M = sp.lil_matrix((n + 2, n + 2))
    for t in range(0, n + 1):
        M[t, t] = 0.5
        M[t, t + 1] = 0.5
    return M.tocsr()


class MacOps:
    def __init__(self, nx, ny, nz, s=0.0):
        self.n = (nx, ny, nz)
        self.s = s
        self.P = (nx + 2) * (ny + 2) * (nz + 2)

    def kron3(self, mats):
        """mats = (Mx, My, Mz) -> operator on the flattened padded array."""
        Mx, My, Mz = mats
        return sp.kron(sp.kron(Mz, My), Mx).tocsr()

    def eye(self, a):
        return sp.identity(self.n[a] + 2, format="csr")

    def along(self, a, M):
        mats = [self.eye(0), self.eye(1), self.eye(2)]
        mats[a] = M
        return self.kron3(mats)

    def laplace(self, F):
        return sum(self.along(a, d2_1d(self.n[a], F == a, self.s)) for a in range(3))

    def deriv(self, F, a):
        return self.along(a, d1_1d(self.n[a], F == a, self.s))

    def interp(self, c, F):
        """Velocity component c (faces normal to axis c) to the nodes of field F (3 = cell)."""
        if c == F:
            return sp.identity(self.P, format="csr")
        mats = [self.eye(0), self.eye(1), self.eye(2)]
        mats[c] = face_to_cell(self.n[c])
        if F < 3:
            mats[F] = cell_to_face(self.n[F])
        return self.kron3(mats)

    def dof_mask(self, F):
        m = []
        for a in range(3):
            v = np.zeros(self.n[a] + 2)
            v[interior_rows(self.n[a], F == a)] = 1.0
            m.append(v)
        return np.kron(np.kron(m[2], m[1]), m[0])

    def upwind_deriv(self, F, a, sel):
        """First derivative along axis a at the nodes of field F, one-sided towards the
        upstream node: backward where the node's selecting velocity sel is >= 0."""
        back = self.along(a, d1_side_1d(self.n[a], F == a, True, self.s))
        fwd = self.along(a, d1_side_1d(self.n[a], F == a, False, self.s))
        pos = (sel >= 0.0).astype(float)
        return sp.diags(pos) @ back + sp.diags(1.0 - pos) @ fwd

    def jacobian(self, base, gr, pr, upwind=False):
        """Sparse J acting on a packed (u, v, w, T) vector already in Eq (13)'s space. With
        upwind, each derivative of an advection term is one-sided, chosen by the sign of the
        base velocity component averaged to the node (in both (U.grad)v and (v.grad)U)."""
        P = self.P
        nu, kappa = gr ** -0.5, 1.0 / (pr * gr ** 0.5)
        Ub = [base[c].ravel() for c in range(3)]
        Th = base[3].ravel()
        blocks = [[None] * 4 for _ in range(4)]
        for F in range(4):
            adv = [self.interp(c, F) @ Ub[c] for c in range(3)]
            D = [self.upwind_deriv(F, c, adv[c]) if upwind else self.deriv(F, c) for c in range(3)]
            diag_adv = sum(sp.diags(adv[c]) @ D[c] for c in range(3))
            coef = kappa if F == 3 else nu
            own = coef * self.laplace(F) - diag_adv
            target = Th if F == 3 else Ub[F]
            for c in range(3):
                # -(x . grad) target: the perturbation velocity averaged, times grad of target
                term = -sp.diags(D[c] @ target) @ self.interp(c, F)
                blocks[F][c] = term if blocks[F][c] is None else blocks[F][c] + term
            blocks[F][F] = own if blocks[F][F] is None else blocks[F][F] + own
            if F == 2:
                blocks[2][3] = self.along(2, cell_to_face(self.n[2]))
        for F in range(4):
            for c in range(4):
                if blocks[F][c] is None:
                    blocks[F][c] = sp.csr_matrix((P, P))
        J = sp.bmat(blocks, format="csr")
        mask = np.concatenate([self.dof_mask(F) for F in range(4)])
        return sp.diags(mask) @ J

    def divergence(self):
        """Cells (padded, interior rows) <- faces; D v with MAC differences."""
        P = self.P
        parts = []
        for a in range(3):
            n = self.n[a]
            w = control_volume(n, False, self.s)
            M = sp.lil_matrix((n + 2, n + 2))
            for t in range(1, n + 1):
                M[t, t] = 1.0 / w[t]
                M[t, t - 1] = -1.0 / w[t]
            parts.append(self.along(a, M.tocsr()))
        D = sp.hstack(parts).tocsr()
        return sp.diags(self.dof_mask(3)) @ D

    def gradient(self):
        """Interior faces <- cells; (G phi)_face = (phi_{t+1} - phi_t) / h."""
        rows = []
        for a in range(3):
            n = self.n[a]
            w = control_volume(n, True, self.s)
            M = sp.lil_matrix((n + 2, n + 2))
            for t in range(1, n):
                M[t, t + 1] = 1.0 / w[t]
                M[t, t] = -1.0 / w[t]
            rows.append(sp.diags(self.dof_mask(a)) @ self.along(a, M.tocsr()))
        return sp.vstack(rows).tocsr()
