"""ctypes wrapper over the plain C FP64 oracle in kv_oracle.c (test infrastructure only).

Every function takes and returns numpy float64 arrays in the padded layout
(nz+2, ny+2, nx+2), x fastest; packed vectors are (4, nz+2, ny+2, nx+2) = (u, v, w, T).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kv_oracle.c")
_LIB = os.path.join(_HERE, "libkv_oracle.so")


def build_oracle(force: bool = False) -> str:
    """Compile kv_oracle.c with gcc (OpenMP) into oracle/libkv_oracle.so.

    KV_ORACLE_LIB names another build of the same source to load instead (the mutation tests
    load deliberately broken copies this way)."""
    override = os.environ.get("KV_ORACLE_LIB")
    if override:
        return override
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("bc", ctypes.c_int), ("tproj", ctypes.c_int),
                ("gr", ctypes.c_double), ("pr", ctypes.c_double),
                ("stretch", ctypes.c_double), ("adv", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_int), ("max_div", ctypes.c_double),
                ("rel_div", ctypes.c_double), ("phi_norm", ctypes.c_double)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        P = ctypes.c_void_p
        D = ctypes.POINTER(ctypes.c_double)
        lib.or_create.restype = P
        lib.or_create.argtypes = [ctypes.POINTER(_Grid)]
        lib.or_destroy.argtypes = [P]
        lib.or_axis_data.argtypes = [P, ctypes.c_int, ctypes.c_int, D]
        for name in ("or_tproj_gram", "or_project_input", "or_divergence", "or_poisson_tpd",
                     "or_residual_raw"):
            getattr(lib, name).argtypes = [P, D, D]
        lib.or_tproj_closed.argtypes = [P, D]
        lib.or_jx_raw.argtypes = [P, D, D, D]
        lib.or_correct.argtypes = [P, D, D, D]
        lib.or_krylov_vector.argtypes = [P, D, D, D, D, ctypes.c_double, ctypes.c_int,
                                         ctypes.POINTER(Stats)]
        lib.or_newton_residual.restype = ctypes.c_double
        lib.or_newton_residual.argtypes = [P, D, D, ctypes.c_double, ctypes.c_int]
        lib.or_arnoldi_step.argtypes = [P, D, D, ctypes.c_int, D, ctypes.c_double, ctypes.c_int]
        lib.or_jt_raw.argtypes = [P, D, D, D]
        lib.or_krylov_adjoint.argtypes = [P, D, D, D, ctypes.c_double, ctypes.c_int]
        lib.or_grad_base.argtypes = [P, D, D, D]
        lib.or_grad_gr.restype = ctypes.c_double
        lib.or_grad_gr.argtypes = [P, D, D]
        _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Oracle:
    """One grid's oracle context (Eqs (15)-(20)'s per-axis data computed once)."""

    def __init__(self, nx, ny, nz, bc=0, gr=1e6, pr=0.71, tproj=0, tol=1e-13, max_passes=10,
                 stretch=0.0, adv=0):
        self.lib = _load()
        self.nx, self.ny, self.nz = nx, ny, nz
        self.bc, self.gr, self.pr, self.tproj = bc, gr, pr, tproj
        self.tol, self.max_passes, self.stretch, self.adv = tol, max_passes, stretch, adv
        self._g = _Grid(nx, ny, nz, bc, tproj, gr, pr, stretch, adv)
        self._c = self.lib.or_create(ctypes.byref(self._g))
        if not self._c:
            raise ValueError("oracle: invalid grid")

    def __del__(self):
        if getattr(self, "_c", None):
            self.lib.or_destroy(self._c)
            self._c = None

    @property
    def shape(self):
        return (self.nz + 2, self.ny + 2, self.nx + 2)

    def _new(self, *lead):
        return np.zeros(tuple(lead) + self.shape)

    @staticmethod
    def _c64(a):
        return np.ascontiguousarray(a, dtype=np.float64)

    # per-axis data ------------------------------------------------------------------
    def axis_data(self, axis, which):
        n = (self.nx, self.ny, self.nz)[axis]
        size = {0: n * n, 1: n * n, 2: n, 3: (n + 2) ** 2, 4: n + 1, 5: n + 2}[which]
        out = np.zeros(size)
        self.lib.or_axis_data(self._c, axis, which, _ptr(out))
        if which in (0, 1):
            return out.reshape(n, n)
        if which == 3:
            return out.reshape(n + 2, n + 2)
        return out

    # pieces -------------------------------------------------------------------------
    def project_input(self, x):
        x = self._c64(x)
        out = self._new(4)
        self.lib.or_project_input(self._c, _ptr(x), _ptr(out))
        return out

    def jx_raw(self, base, xp):
        base, xp = self._c64(base), self._c64(xp)
        out = self._new(4)
        self.lib.or_jx_raw(self._c, _ptr(base), _ptr(xp), _ptr(out))
        return out

    def residual_raw(self, S):
        S = self._c64(S)
        out = self._new(4)
        self.lib.or_residual_raw(self._c, _ptr(S), _ptr(out))
        return out

    def divergence(self, vel):
        vel = self._c64(vel)
        b = np.zeros((self.nz, self.ny, self.nx))
        self.lib.or_divergence(self._c, _ptr(vel), _ptr(b))
        return b

    def poisson(self, b):
        b = self._c64(b)
        phi = np.zeros((self.nz, self.ny, self.nx))
        self.lib.or_poisson_tpd(self._c, _ptr(b), _ptr(phi))
        return phi

    def correct(self, phi, vel, p=None):
        phi = self._c64(phi)
        vel = self._c64(vel).copy()
        pp = None if p is None else self._c64(p).copy()
        self.lib.or_correct(self._c, _ptr(phi), _ptr(vel), _ptr(pp))
        return vel, pp

    def tproj_gram(self, T):
        T = self._c64(T)
        out = self._new()
        self.lib.or_tproj_gram(self._c, _ptr(T), _ptr(out))
        return out

    def tproj_closed(self, T):
        out = self._c64(T).copy()
        self.lib.or_tproj_closed(self._c, _ptr(out))
        return out

    # the path -----------------------------------------------------------------------
    def krylov_vector(self, base, x, want_p=False, stats=False):
        base, x = self._c64(base), self._c64(x)
        y = self._new(4)
        p = self._new() if want_p else None
        st = Stats()
        self.lib.or_krylov_vector(self._c, _ptr(base), _ptr(x), _ptr(y), _ptr(p), self.tol,
                                  self.max_passes, ctypes.byref(st))
        res = [y]
        if want_p:
            res.append(p)
        if stats:
            res.append(st)
        return res[0] if len(res) == 1 else tuple(res)

    def newton_residual(self, S):
        S = self._c64(S)
        F = self._new(4)
        nrm = self.lib.or_newton_residual(self._c, _ptr(S), _ptr(F), self.tol, self.max_passes)
        return F, nrm

    def arnoldi_step(self, base, V, j):
        """V: (>= j+2, 4, ...) array, modified in place (slot j+1); returns h[0..j+1]."""
        base = self._c64(base)
        assert V.dtype == np.float64 and V.flags.c_contiguous and V.shape[0] >= j + 2
        h = np.zeros(j + 2)
        self.lib.or_arnoldi_step(self._c, _ptr(base), _ptr(V), j, _ptr(h), self.tol,
                                 self.max_passes)
        return h

    # adjoint ------------------------------------------------------------------------
    def jt_raw(self, base, ys):
        base, ys = self._c64(base), self._c64(ys)
        z = self._new(4)
        self.lib.or_jt_raw(self._c, _ptr(base), _ptr(ys), _ptr(z))
        return z

    def krylov_adjoint(self, base, y):
        """z = A^T y (orthogonal reading of the temperature projection)."""
        assert self.tproj == 0, "the transpose is defined for the orthogonal reading"
        base, y = self._c64(base), self._c64(y)
        z = self._new(4)
        self.lib.or_krylov_adjoint(self._c, _ptr(base), _ptr(y), _ptr(z), self.tol, self.max_passes)
        return z

    def grad_base(self, xp, ys):
        """d <ys, J(base) xp> / d base, a packed (U, V, W, Theta) array."""
        xp, ys = self._c64(xp), self._c64(ys)
        g = self._new(4)
        self.lib.or_grad_base(self._c, _ptr(xp), _ptr(ys), _ptr(g))
        return g

    def grad_gr(self, xp, ys):
        xp, ys = self._c64(xp), self._c64(ys)
        return self.lib.or_grad_gr(self._c, _ptr(xp), _ptr(ys))
