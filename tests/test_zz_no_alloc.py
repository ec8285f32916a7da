"""The allocation-free entry point kv_krylov_vector_noalloc, for callers that cannot allocate
device memory (it uses a fixed __device__ scratch array instead of library buffers).

Checked through the C ABI against the handle-based kv_krylov_vector on two calls in a row,
within the FP64 tolerance of the other parity tests. This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_1905_11601_gb300 import synth

pytestmark = pytest.mark.gpu
RTOL = 1e-12
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_11601_gb300 import build
    build.build()


def _desc(kv, n, bc, gr, precision=0, tproj=0):
    return kv.GridDesc(n[0], n[1], n[2], bc, tproj, precision, gr, 0.71, 0.0, 0, 0, 0)


@pytest.mark.parametrize("n,bc,tproj", [((20, 17, 24), synth.CC, 0), ((32, 9, 30), synth.AA, 0),
                                        ((15, 22, 11), synth.AA, 1)])
def test_noalloc_matches_handle_path_on_two_calls(n, bc, tproj):
    from paper_1905_11601_gb300 import kv
    lib = kv.load_library()
    gr = 2.0e6
    base = torch.from_numpy(np.stack(synth.base_flow(*n, bc, 31))).cuda()
    xs = torch.from_numpy(synth.krylov_input(*n, 32, count=2)).cuda()
    g = kv.Grid(*n, bc=bc, gr=gr, tproj=tproj)
    g.set_base_flow(base)
    desc = _desc(kv, n, bc, gr, tproj=tproj)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        x = xs[call].contiguous()
        y_ref = g.krylov_vector(x)
        y = torch.full_like(x, float("nan"))
        st = lib.kv_krylov_vector_noalloc(ctypes.byref(desc), base.data_ptr(), x.data_ptr(), y.data_ptr(),
                                          ctypes.c_void_p(stream))
        assert st == 0, lib.kv_last_error(None)
        torch.cuda.synchronize()
        err = (torch.linalg.vector_norm(y - y_ref) / torch.linalg.vector_norm(y_ref)).item()
        assert err < RTOL, (call, err)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1905_11601_gb300 import kv
    lib = kv.load_library()
    n = (33, 8, 8)
    t = torch.zeros((4, 10, 10, 35), dtype=torch.float64, device="cuda")
    y = torch.zeros_like(t)
    st = lib.kv_krylov_vector_noalloc(ctypes.byref(_desc(kv, n, 0, 1e6)), t.data_ptr(), t.data_ptr(),
                                      y.data_ptr(), None)
    assert st == -1
    assert b"32" in lib.kv_last_error(None)
    st = lib.kv_krylov_vector_noalloc(ctypes.byref(_desc(kv, (8, 8, 8), 0, 1e6, precision=1)), t.data_ptr(),
                                      t.data_ptr(), y.data_ptr(), None)
    assert st == -1
    # a base state overlapping y is refused (the operator reads base while y is written)
    n = (8, 8, 8)
    buf = torch.zeros((2, 4, 10, 10, 10), dtype=torch.float64, device="cuda")
    st = lib.kv_krylov_vector_noalloc(ctypes.byref(_desc(kv, n, 0, 1e6)), buf[1].data_ptr(), buf[0].data_ptr(),
                                      buf[1].data_ptr(), None)
    assert st == -1
    assert b"overlap" in lib.kv_last_error(None)
