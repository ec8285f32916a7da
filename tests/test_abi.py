"""The C-ABI library: it loads, exports every symbol include/kv.h declares, and rejects bad
descriptors on the host before any CUDA call (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_1905_11601_gb300 import build as kvbuild
from paper_1905_11601_gb300 import kv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    kvbuild.build()
    return kv.load_library()


def declared_functions():
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if hdr.endswith(".h"):
            text = open(os.path.join(ROOT, "include", hdr)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(kv_[a-z0-9_]+)\s*\(", text))
    return names


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert {"kv_create_grid", "kv_krylov_vector", "kv_arnoldi_step", "kv_newton_residual",
            "kv_set_base_flow"} <= names
    for n in names:
        assert hasattr(lib, n), n
    assert set(kv.EXPORTS) <= names


def _desc(**kw):
    d = dict(nx=8, ny=8, nz=8, spanwise_bc=0, tproj=0, precision=0, gr=1e6, pr=0.71, tol=0.0, max_passes=0,
             refine_sweeps=0, cgs_passes=0, stretch=0.0)
    d.update(kw)
    return kv.GridDesc(**d)


@pytest.mark.parametrize("bad", [dict(nx=1), dict(nz=2000), dict(spanwise_bc=3), dict(tproj=7),
                                 dict(precision=9), dict(gr=-1.0), dict(pr=0.0), dict(max_passes=-1),
                                 dict(gr=float("nan")), dict(refine_sweeps=-1), dict(refine_sweeps=99), dict(cgs_passes=1),
                                 dict(stretch=-0.01), dict(stretch=0.16), dict(stretch=float("nan")),
                                 dict(advection=2), dict(advection=-1), dict(advection=1, stretch=0.05)])
def test_invalid_descriptor_rejected_on_host(lib, bad):
    h = ctypes.c_void_p()
    st = lib.kv_create_grid(ctypes.byref(_desc(**bad)), None, ctypes.byref(h))
    assert st == -1 and not h.value
    assert lib.kv_last_error(None)


def test_stretched_grid_rejected_by_the_allocation_free_entry(lib):
    # validated on the host before any device call
    d = _desc(stretch=0.05)
    buf = (ctypes.c_double * 8)()
    assert lib.kv_krylov_vector_noalloc(ctypes.byref(d), buf, buf, buf, None) == -1


def test_upwind_rejected_by_the_allocation_free_entry(lib):
    d = _desc(advection=kv.KV_ADV_UPWIND)
    buf = (ctypes.c_double * 8)()
    assert lib.kv_krylov_vector_noalloc(ctypes.byref(d), buf, buf, buf, None) == -1
    assert b"central" in lib.kv_last_error(None)


def test_null_arguments_rejected(lib):
    assert lib.kv_create_grid(None, None, None) == -1
    assert lib.kv_destroy_grid(None) == 0
    assert lib.kv_krylov_vector(None, None, None, None, None) == -1
    assert lib.kv_arnoldi_step(None, None, 0, None) == -1
    assert lib.kv_arnoldi_run(None, None, 0, 1, None, 2) == -1
    assert lib.kv_newton_residual(None, None, None, None) == -1
    assert lib.kv_set_base_flow(None, None, None, None, None) == -1
    assert lib.kv_set_base_flow_packed(None, None) == -1
    assert lib.kv_field_sizes(None, None, None, None, None) == -1
    assert lib.kv_set_tuning(None, None) == -1
    assert lib.kv_guard_read(None, None, 0) == -1
    assert lib.kv_arnoldi_counts(None, None, None) == -1
    assert lib.kv_krylov_vector_host(None, None, None, None) == -1
    assert lib.kv_krylov_vector_host_stream(None, None, None, 1) == -1
    assert lib.kv_gmres(None, None, None, None, 10, 1, 1e-10, 0.99, None) == -1
    assert lib.kv_bicgstab2(None, None, None, None, 10, 1e-10, None) == -1
    assert lib.kv_newton(None, None, None, None, None, None) == -1
    assert lib.kv_axpby(None, 1.0, None, 1.0, None) == -1
    assert lib.kv_combine(None, None, 1, None, None) == -1
    out = ctypes.c_double()
    assert lib.kv_dot(None, None, None, ctypes.byref(out)) == -1
