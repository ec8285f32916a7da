"""Python binding of libkv (include/kv.h): argument marshalling only.

Every step of the Krylov-vector evaluation runs in the CUDA kernels of libkv.so; torch is
used for device memory and streams. There is no CPU fallback: if the library is missing or
no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libkv.so")

KV_BC_CC, KV_BC_AA = 0, 1
KV_TPROJ_ORTHOGONAL, KV_TPROJ_OBLIQUE = 0, 1
KV_PREC_FP64, KV_PREC_MIXED = 0, 1
KV_ADV_CENTRAL, KV_ADV_UPWIND = 0, 1

_STATUS = {0: "KV_OK", -1: "KV_ERR_ARG", -2: "KV_ERR_CUDA", -3: "KV_ERR_NOT_CONVERGED", -4: "KV_ERR_STATE",
           -5: "KV_ERR_NOMEM"}

# every symbol include/kv.h declares
EXPORTS = ("kv_create_grid", "kv_destroy_grid", "kv_set_stream", "kv_field_len", "kv_set_base_flow",
           "kv_krylov_vector", "kv_krylov_vector_host", "kv_arnoldi_step", "kv_arnoldi_run", "kv_newton_residual",
           "kv_last_error",
           "kv_profile_enable", "kv_profile_get", "kv_krylov_vector_noalloc", "kv_krylov_vector_adjoint",
           "kv_base_flow_gradient", "kv_krylov_vector_batch", "kv_plan_create", "kv_plan_add", "kv_plan_launch",
           "kv_plan_destroy", "kv_plan_last_error", "kv_selftest_wait_timeout", "kv_tuning",
           "kv_krylov_vector_host_stream", "kv_gmres", "kv_bicgstab2", "kv_newton", "kv_axpby", "kv_combine", "kv_dot",
           "kv_axis_data", "kv_field_sizes", "kv_set_base_flow_packed", "kv_set_tuning", "kv_guard_read",
           "kv_arnoldi_counts", "kv_set_contraction_tile", "kv_contraction_tile")
PHASES = {"stencil": 0, "divergence": 1, "tpd": 2, "correct": 3, "arnoldi": 4, "refine": 5, "gs_dots": 6,
          "gs_update": 7}


def axis_data(n, stretch=0.0):
    """kv_axis_data on the host (no CUDA call): (E, E_inv, lambda, weights) of one axis of n cells,
    as numpy arrays of shapes (n, n), (n, n), (n,) and (14, n + 2); see include/kv.h."""
    lib = load_library()
    E, Ei = np.zeros((n, n)), np.zeros((n, n))
    lam, w = np.zeros(n), np.zeros((14, n + 2))
    P = ctypes.POINTER(ctypes.c_double)
    st = lib.kv_axis_data(n, stretch, *(a.ctypes.data_as(P) for a in (E, Ei, lam, w)))
    if st != 0:
        raise KvError(st, lib.kv_last_error(None).decode())
    return E, Ei, lam, w


class KvError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class GridDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("spanwise_bc", ctypes.c_int), ("tproj", ctypes.c_int), ("precision", ctypes.c_int),
                ("gr", ctypes.c_double), ("pr", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_passes", ctypes.c_int), ("refine_sweeps", ctypes.c_int), ("cgs_passes", ctypes.c_int),
                ("stretch", ctypes.c_double), ("advection", ctypes.c_int)]


class Guard(ctypes.Structure):
    """kv_guard: the device-side SIMPLE test of the one-pass evaluations."""
    _fields_ = [("checks", ctypes.c_longlong), ("failed", ctypes.c_longlong), ("nonfinite", ctypes.c_longlong),
                ("worst_rel_div", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_int), ("max_div", ctypes.c_double), ("rel_div", ctypes.c_double),
                ("refine_residual", ctypes.c_double), ("device_error", ctypes.c_int)]


class SolveStats(ctypes.Structure):
    """kv_solve_stats of kv_gmres / kv_bicgstab2."""
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int), ("matvecs", ctypes.c_int),
                ("converged", ctypes.c_int), ("saturated", ctypes.c_int), ("breakdown", ctypes.c_int),
                ("rel_residual", ctypes.c_double)]


NEWTON_HISTORY = 64


class NewtonParams(ctypes.Structure):
    _fields_ = [("max_newton", ctypes.c_int), ("tol", ctypes.c_double), ("gmres_m", ctypes.c_int),
                ("gmres_max_restarts", ctypes.c_int), ("lin_tol", ctypes.c_double), ("gmres_sat", ctypes.c_double),
                ("bicg_max_iter", ctypes.c_int)]


class NewtonStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("matvecs", ctypes.c_int), ("gmres_restarts", ctypes.c_int),
                ("bicg_iterations", ctypes.c_int), ("bicg_rejected", ctypes.c_int), ("converged", ctypes.c_int),
                ("n_res", ctypes.c_int),
                ("res_norm", ctypes.c_double * NEWTON_HISTORY)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libkv.so and declares its signatures (no CUDA call is made)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libkv.so not built ({path}); run paper_1905_11601_gb300.build.build()")
    lib = ctypes.CDLL(path)
    H = ctypes.c_void_p
    D = ctypes.c_void_p  # device or host pointer (int address)
    lib.kv_create_grid.argtypes = [ctypes.POINTER(GridDesc), ctypes.c_void_p, ctypes.POINTER(H)]
    lib.kv_destroy_grid.argtypes = [H]
    lib.kv_set_stream.argtypes = [H, ctypes.c_void_p]
    lib.kv_field_len.argtypes = [H, ctypes.POINTER(ctypes.c_size_t)]
    lib.kv_set_base_flow.argtypes = [H, D, D, D, D]
    lib.kv_set_base_flow_packed.argtypes = [H, D]
    S = ctypes.POINTER(ctypes.c_size_t)
    lib.kv_field_sizes.argtypes = [H, S, S, S, S]
    lib.kv_set_tuning.argtypes = [H, ctypes.POINTER(ctypes.c_int)]
    lib.kv_set_contraction_tile.argtypes = [H, ctypes.c_int]
    lib.kv_contraction_tile.argtypes = [H, ctypes.POINTER(ctypes.c_int)]
    lib.kv_guard_read.argtypes = [H, ctypes.POINTER(Guard), ctypes.c_int]
    lib.kv_arnoldi_counts.argtypes = [H, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
    lib.kv_krylov_vector.argtypes = [H, D, D, D, ctypes.POINTER(Stats)]
    lib.kv_krylov_vector_host.argtypes = [H, D, D, ctypes.POINTER(Stats)]
    lib.kv_arnoldi_step.argtypes = [H, D, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    lib.kv_arnoldi_run.argtypes = [H, D, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    lib.kv_newton_residual.argtypes = [H, D, D, ctypes.POINTER(ctypes.c_double)]
    lib.kv_profile_enable.argtypes = [H, ctypes.c_int]
    lib.kv_profile_get.argtypes = [H, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
    lib.kv_tuning.argtypes = [H, ctypes.POINTER(ctypes.c_int)]
    lib.kv_krylov_vector_host_stream.argtypes = [H, D, D, ctypes.c_int]
    lib.kv_gmres.argtypes = [H, D, D, D, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                             ctypes.POINTER(SolveStats)]
    lib.kv_bicgstab2.argtypes = [H, D, D, D, ctypes.c_int, ctypes.c_double, ctypes.POINTER(SolveStats)]
    lib.kv_newton.argtypes = [H, D, D, D, ctypes.POINTER(NewtonParams), ctypes.POINTER(NewtonStats)]
    lib.kv_axpby.argtypes = [H, ctypes.c_double, D, ctypes.c_double, D]
    lib.kv_combine.argtypes = [H, D, ctypes.c_int, ctypes.POINTER(ctypes.c_double), D]
    lib.kv_dot.argtypes = [H, D, D, ctypes.POINTER(ctypes.c_double)]
    P = ctypes.POINTER(ctypes.c_double)
    lib.kv_axis_data.argtypes = [ctypes.c_int, ctypes.c_double, P, P, P, P]
    lib.kv_krylov_vector_adjoint.argtypes = [H, D, D]
    lib.kv_base_flow_gradient.argtypes = [H, D, D, D, ctypes.POINTER(ctypes.c_double)]
    lib.kv_krylov_vector_batch.argtypes = [H, D, D, ctypes.c_int]
    lib.kv_plan_create.argtypes = [ctypes.POINTER(ctypes.c_void_p)]
    lib.kv_plan_add.argtypes = [ctypes.c_void_p, H, D, D]
    lib.kv_plan_launch.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.kv_plan_destroy.argtypes = [ctypes.c_void_p]
    lib.kv_plan_last_error.argtypes = [ctypes.c_void_p]
    lib.kv_plan_last_error.restype = ctypes.c_char_p
    lib.kv_selftest_wait_timeout.argtypes = [H, ctypes.POINTER(ctypes.c_int)]
    lib.kv_krylov_vector_noalloc.argtypes = [ctypes.POINTER(GridDesc), D, D, D, ctypes.c_void_p]
    lib.kv_last_error.argtypes = [H]
    lib.kv_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("kv_last_error", "kv_plan_last_error"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _dev_ptr(t, torch, name, numel=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous float64 CUDA tensor")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name}: needs at least {numel} elements, got {t.numel()}")
    return t.data_ptr()


class Grid:
    """A grid handle: kv_create_grid / kv_destroy_grid around the calls of include/kv.h."""

    def __init__(self, nx, ny, nz, bc=KV_BC_CC, gr=1.0e6, pr=0.71, tproj=KV_TPROJ_ORTHOGONAL,
                 precision=KV_PREC_FP64, tol=0.0, max_passes=0, refine_sweeps=0, cgs_passes=0, stretch=0.0,
                 advection=0):
        import torch

        self.torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("libkv needs a CUDA device")
        self.lib = load_library()
        self.nx, self.ny, self.nz = nx, ny, nz
        self.desc = GridDesc(nx, ny, nz, bc, tproj, precision, gr, pr, tol, max_passes, refine_sweeps, cgs_passes,
                             stretch, advection)
        h = ctypes.c_void_p()
        st = self.lib.kv_create_grid(ctypes.byref(self.desc), ctypes.c_void_p(self._stream()), ctypes.byref(h))
        if st != 0:
            raise KvError(st, self.lib.kv_last_error(None).decode())
        self.h = h
        n = ctypes.c_size_t()
        self._check(self.lib.kv_field_len(self.h, ctypes.byref(n)))
        self.field_len = n.value
        self.shape = (nz + 2, ny + 2, nx + 2)

    def _stream(self):
        return self.torch.cuda.current_stream().cuda_stream

    def _check(self, st):
        if st != 0:
            raise KvError(st, self.lib.kv_last_error(self.h).decode())

    def _sync_stream(self):
        self._check(self.lib.kv_set_stream(self.h, ctypes.c_void_p(self._stream())))

    def close(self):
        if getattr(self, "h", None):
            self.lib.kv_destroy_grid(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty(self, *lead):
        return self.torch.zeros(tuple(lead) + self.shape, dtype=self.torch.float64, device="cuda")

    def set_base_flow(self, base):
        """base: a packed state U | V | W | Theta (CUDA float64), passed field by field to
        kv_set_base_flow."""
        self._sync_stream()
        P = self.field_len
        p = _dev_ptr(base, self.torch, "base", 4 * P)
        self._check(self.lib.kv_set_base_flow(self.h, p, p + 8 * P, p + 16 * P, p + 24 * P))

    def set_base_flow_fields(self, U, V, W, Theta):
        """The four fields as separate CUDA float64 tensors of one padded field each."""
        self._sync_stream()
        P = self.field_len
        self._check(self.lib.kv_set_base_flow(self.h, *(_dev_ptr(f, self.torch, n, P) for f, n in
                                                        ((U, "U"), (V, "V"), (W, "W"), (Theta, "Theta")))))

    def set_base_flow_packed(self, base):
        self._sync_stream()
        self._check(self.lib.kv_set_base_flow_packed(self.h, _dev_ptr(base, self.torch, "base", 4 * self.field_len)))

    def field_sizes(self):
        """kv_field_sizes: padded lengths of the u, v, w and cell fields."""
        out = [ctypes.c_size_t() for _ in range(4)]
        self._check(self.lib.kv_field_sizes(self.h, *(ctypes.byref(o) for o in out)))
        return tuple(o.value for o in out)

    def set_tuning(self, apply_block=(32, 8), df_variant=-1, df_block=(-1, -1)):
        """kv_set_tuning: fix the operator configuration (same layout as tuning())."""
        cfg = (ctypes.c_int * 5)(apply_block[0], apply_block[1], df_variant, df_block[0], df_block[1])
        self._check(self.lib.kv_set_tuning(self.h, cfg))

    def guard(self, reset=False):
        """kv_guard_read: {checks, failed, nonfinite, worst_rel_div} of the device-side SIMPLE test."""
        self._sync_stream()
        g = Guard()
        self._check(self.lib.kv_guard_read(self.h, ctypes.byref(g), 1 if reset else 0))
        return {"checks": g.checks, "failed": g.failed, "nonfinite": g.nonfinite, "worst_rel_div": g.worst_rel_div}

    def arnoldi_counts(self):
        """(fused Arnoldi steps, of them with the second Gram-Schmidt update) since profile_enable."""
        a, b = ctypes.c_longlong(), ctypes.c_longlong()
        self._check(self.lib.kv_arnoldi_counts(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def krylov_vector(self, x, y=None, p=None, stats=False):
        self._sync_stream()
        if y is None:
            y = self.empty(4)
        st = Stats()
        self._check(self.lib.kv_krylov_vector(self.h, _dev_ptr(x, self.torch, "x", 4 * self.field_len),
                                              _dev_ptr(y, self.torch, "y", 4 * self.field_len),
                                              _dev_ptr(p, self.torch, "p", self.field_len),
                                              ctypes.byref(st) if stats else None))
        return (y, st) if stats else y

    def krylov_vector_host(self, x_host, y_host, stats=False):
        """x_host, y_host: host float64 arrays/tensors (pinned recommended), 4 packed fields."""
        self._sync_stream()

        def hp(a, name):
            if isinstance(a, np.ndarray):
                assert a.dtype == np.float64 and a.flags.c_contiguous and a.size >= 4 * self.field_len, name
                return a.ctypes.data
            assert not a.is_cuda and a.dtype == self.torch.float64 and a.is_contiguous(), name
            assert a.numel() >= 4 * self.field_len, name
            return a.data_ptr()

        st = Stats()
        self._check(self.lib.kv_krylov_vector_host(self.h, hp(x_host, "x_host"), hp(y_host, "y_host"),
                                                   ctypes.byref(st) if stats else None))
        return st if stats else None

    def krylov_vector_host_stream(self, X_host, Y_host):
        """Y[i] = A X[i] for host float64 tensors/arrays of shape (nb, 4 packed fields) (pinned
        for the copies to overlap the evaluations)."""
        self._sync_stream()
        L = 4 * self.field_len

        def hp(a, name):
            if isinstance(a, np.ndarray):
                assert a.dtype == np.float64 and a.flags.c_contiguous and a.size % L == 0, name
                return a.ctypes.data, a.size // L
            assert not a.is_cuda and a.dtype == self.torch.float64 and a.is_contiguous(), name
            assert a.numel() % L == 0, name
            return a.data_ptr(), a.numel() // L

        px, nb = hp(X_host, "X_host")
        py, nby = hp(Y_host, "Y_host")
        assert nb == nby, "X_host and Y_host hold different numbers of vectors"
        self._check(self.lib.kv_krylov_vector_host_stream(self.h, px, py, nb))

    def gmres(self, b, x, V, m, max_restarts, tol, sat=0.99):
        """Restarted GMRES(m) for A x = b (kv_gmres): x in-out, V an (m + 1)-vector workspace
        (CUDA float64 tensors). Returns SolveStats."""
        self._sync_stream()
        L = 4 * self.field_len
        st = SolveStats()
        self._check(self.lib.kv_gmres(self.h, _dev_ptr(b, self.torch, "b", L), _dev_ptr(x, self.torch, "x", L),
                                      _dev_ptr(V, self.torch, "V", (m + 1) * L), m, max_restarts, tol, sat,
                                      ctypes.byref(st)))
        return st

    def bicgstab2(self, b, x, work, max_iter, tol):
        """BiCGstab(2) for A x = b (kv_bicgstab2): x in-out, work an 8-vector workspace. Returns
        SolveStats."""
        self._sync_stream()
        L = 4 * self.field_len
        st = SolveStats()
        self._check(self.lib.kv_bicgstab2(self.h, _dev_ptr(b, self.torch, "b", L), _dev_ptr(x, self.torch, "x", L),
                                          _dev_ptr(work, self.torch, "work", 8 * L), max_iter, tol,
                                          ctypes.byref(st)))
        return st

    def newton(self, S, V, work, max_newton=10, tol=1e-10, gmres_m=100, gmres_max_restarts=40, lin_tol=1e-10,
               gmres_sat=0.99, bicg_max_iter=1000):
        """Newton's method for the steady state (kv_newton): S in-out (packed state with its wall
        values), V an (m + 1)-vector and work a 10-vector workspace. Returns NewtonStats."""
        self._sync_stream()
        L = 4 * self.field_len
        prm = NewtonParams(max_newton, tol, gmres_m, gmres_max_restarts, lin_tol, gmres_sat, bicg_max_iter)
        st = NewtonStats()
        self._check(self.lib.kv_newton(self.h, _dev_ptr(S, self.torch, "S", L),
                                       _dev_ptr(V, self.torch, "V", (gmres_m + 1) * L),
                                       _dev_ptr(work, self.torch, "work", 10 * L), ctypes.byref(prm),
                                       ctypes.byref(st)))
        return st

    def axpby(self, a, x, b, y):
        """y = a x + b y on packed vectors (kv_axpby)."""
        self._sync_stream()
        L = 4 * self.field_len
        self._check(self.lib.kv_axpby(self.h, float(a), _dev_ptr(x, self.torch, "x", L), float(b),
                                      _dev_ptr(y, self.torch, "y", L)))

    def dot(self, x, y):
        """<x, y> over the packed entries (kv_dot)."""
        self._sync_stream()
        L = 4 * self.field_len
        out = ctypes.c_double()
        self._check(self.lib.kv_dot(self.h, _dev_ptr(x, self.torch, "x", L), _dev_ptr(y, self.torch, "y", L),
                                    ctypes.byref(out)))
        return out.value

    def combine(self, V, c, y):
        """y = sum_i c[i] V[i] over the first len(c) packed vectors of V (kv_combine)."""
        self._sync_stream()
        L = 4 * self.field_len
        c = np.ascontiguousarray(c, dtype=np.float64)
        self._check(self.lib.kv_combine(self.h, _dev_ptr(V, self.torch, "V", len(c) * L), len(c),
                                        c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        _dev_ptr(y, self.torch, "y", L)))

    def arnoldi_run(self, V, j0, m, H=None):
        """kv_arnoldi_run: m Arnoldi steps from the orthonormal V[0..j0] (delayed classical
        Gram-Schmidt). H: the Hessenberg matrix so far (at least j0 columns used), or None when
        j0 == 0. Returns the (j0 + m + 1) x (j0 + m) Hessenberg matrix (numpy)."""
        import numpy as np

        self._sync_stream()
        J = j0 + m
        Hf = np.zeros((J + 1, J), order="F")
        if H is not None and j0 > 0:
            H = np.asarray(H, dtype=np.float64)
            Hf[: min(H.shape[0], J + 1), :j0] = H[: J + 1, :j0]
        L = 4 * self.field_len
        self._check(self.lib.kv_arnoldi_run(self.h, _dev_ptr(V, self.torch, "V", (J + 1) * L), j0, m,
                                            Hf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), J + 1))
        return np.ascontiguousarray(Hf)

    def arnoldi_step(self, V, j):
        self._sync_stream()
        L = 4 * self.field_len
        hcol = (ctypes.c_double * (j + 2))()
        self._check(self.lib.kv_arnoldi_step(self.h, _dev_ptr(V, self.torch, "V", (j + 2) * L), j, hcol))
        return np.array(hcol[:])

    def krylov_vector_batch(self, X, Y=None):
        """Y[b] = A X[b] for a block X of shape (nb, 4, nz+2, ny+2, nx+2), replayed from a CUDA graph."""
        self._sync_stream()
        nb = X.shape[0]
        if Y is None:
            Y = self.empty(nb, 4)
        self._check(self.lib.kv_krylov_vector_batch(self.h, _dev_ptr(X, self.torch, "X", nb * 4 * self.field_len),
                                                    _dev_ptr(Y, self.torch, "Y", nb * 4 * self.field_len), nb))
        return Y

    def krylov_vector_adjoint(self, y, z=None):
        """z = A^T y (transpose of the Krylov map)."""
        self._sync_stream()
        if z is None:
            z = self.empty(4)
        self._check(self.lib.kv_krylov_vector_adjoint(self.h, _dev_ptr(y, self.torch, "y", 4 * self.field_len),
                                                      _dev_ptr(z, self.torch, "z", 4 * self.field_len)))
        return z

    def base_flow_gradient(self, x, y, want_base=True, want_gr=True):
        """(d<y, A x>/d(U, V, W, Theta) as a packed state or None, d<y, A x>/d Gr or None)."""
        self._sync_stream()
        gt = self.empty(4) if want_base else None
        dgr = ctypes.c_double()
        self._check(self.lib.kv_base_flow_gradient(self.h, _dev_ptr(x, self.torch, "x", 4 * self.field_len),
                                                   _dev_ptr(y, self.torch, "y", 4 * self.field_len),
                                                   _dev_ptr(gt, self.torch, "g_base", 4 * self.field_len),
                                                   ctypes.byref(dgr) if want_gr else None))
        return gt, (dgr.value if want_gr else None)

    def selftest_wait_timeout(self):
        """Runs the bounded-wait expiry self-test; returns the device error flag it produced."""
        self._sync_stream()
        de = ctypes.c_int()
        self._check(self.lib.kv_selftest_wait_timeout(self.h, ctypes.byref(de)))
        return de.value

    def profile_enable(self, on=True):
        self._sync_stream()
        self._check(self.lib.kv_profile_enable(self.h, 1 if on else 0))

    def tuning(self):
        """The autotuner's choice: {"apply_block": (bx, by), "df_variant": 0 split + per-equation
        kernel | 1 double-float march | 2 fixed-point march | -1 (FP64 grid), "df_block": (cells,
        rows) | (0, planes per block), "contraction_tile": 256 | 128 | -1 (FP64 grid)}."""
        cfg = (ctypes.c_int * 5)()
        self._check(self.lib.kv_tuning(self.h, cfg))
        return {"apply_block": (cfg[0], cfg[1]), "df_variant": cfg[2], "df_block": (cfg[3], cfg[4]),
                "contraction_tile": self.contraction_tile()}

    def set_contraction_tile(self, columns):
        """kv_set_contraction_tile: 256 or 128 output columns per tensor-core tile."""
        self._check(self.lib.kv_set_contraction_tile(self.h, int(columns)))

    def contraction_tile(self):
        c = ctypes.c_int()
        self._check(self.lib.kv_contraction_tile(self.h, ctypes.byref(c)))
        return c.value

    def profile(self):
        """{phase: (total_ms, timed_brackets, launches)} since the last profile_enable."""
        out = {}
        for name, ph in PHASES.items():
            ms, nt, nl = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_longlong()
            self._check(self.lib.kv_profile_get(self.h, ph, ctypes.byref(ms), ctypes.byref(nt), ctypes.byref(nl)))
            out[name] = (ms.value, nt.value, nl.value)
        return out

    def newton_residual(self, S, F=None):
        self._sync_stream()
        if F is None:
            F = self.empty(4)
        nrm = ctypes.c_double()
        self._check(self.lib.kv_newton_residual(self.h, _dev_ptr(S, self.torch, "S", 4 * self.field_len),
                                                _dev_ptr(F, self.torch, "F", 4 * self.field_len),
                                                ctypes.byref(nrm)))
        return F, nrm.value


class Plan:
    """Several grids' Krylov vectors evaluated by one CUDA-graph launch (kv_plan_*)."""

    def __init__(self):
        import torch

        self.torch = torch
        self.lib = load_library()
        p = ctypes.c_void_p()
        st = self.lib.kv_plan_create(ctypes.byref(p))
        if st != 0:
            raise KvError(st, "kv_plan_create")
        self.p = p
        self._keep = []

    def add(self, grid, x, y):
        st = self.lib.kv_plan_add(self.p, grid.h, _dev_ptr(x, self.torch, "x", 4 * grid.field_len),
                                  _dev_ptr(y, self.torch, "y", 4 * grid.field_len))
        if st != 0:
            raise KvError(st, self.lib.kv_plan_last_error(self.p).decode())
        self._keep.append((grid, x, y))

    def launch(self):
        st = self.lib.kv_plan_launch(self.p, ctypes.c_void_p(self.torch.cuda.current_stream().cuda_stream))
        if st != 0:
            raise KvError(st, self.lib.kv_plan_last_error(self.p).decode())

    def close(self):
        if getattr(self, "p", None):
            self.lib.kv_plan_destroy(self.p)
            self.p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
