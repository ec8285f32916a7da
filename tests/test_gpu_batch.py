"""Batched evaluation replayed from a CUDA graph, and multi-grid plans (several grids, Grashof
numbers and boundary types in one graph launch): results equal the single-vector path."""
import numpy as np
import pytest

from paper_1905_11601_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_11601_gb300 import build
    build.build()


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_single_calls_and_replays(precision):
    from paper_1905_11601_gb300 import kv
    n = (24, 20, 18)
    g = kv.Grid(*n, gr=2e6, precision=precision)
    g.set_base_flow(torch.from_numpy(np.stack(synth.base_flow(*n, synth.CC, 101))).cuda())
    X = torch.from_numpy(synth.krylov_input(*n, 102, count=5)).cuda()
    ref = torch.stack([g.krylov_vector(X[b].contiguous()) for b in range(5)])
    Y = g.krylov_vector_batch(X)
    torch.cuda.synchronize()
    assert torch.equal(Y, ref)
    # replay with new contents of the same buffers
    X.copy_(torch.from_numpy(synth.krylov_input(*n, 103, count=5)))
    g.krylov_vector_batch(X, Y)
    ref = torch.stack([g.krylov_vector(X[b].contiguous()) for b in range(5)])
    torch.cuda.synchronize()
    assert torch.equal(Y, ref)


def test_plan_over_mixed_grids():
    """Grids of different sizes, boundary types, Grashof numbers and precisions in one graph."""
    from paper_1905_11601_gb300 import kv
    specs = [((16, 16, 16), synth.CC, 1e6, 0), ((20, 12, 18), synth.AA, 4e6, 0), ((32, 32, 32), synth.CC, 2e6, 1),
             ((24, 24, 24), synth.AA, 3e6, 1)]
    plan = kv.Plan()
    grids, xs, ys, refs = [], [], [], []
    for q, (n, bc, gr, prec) in enumerate(specs):
        g = kv.Grid(*n, bc=bc, gr=gr, precision=prec)
        g.set_base_flow(torch.from_numpy(np.stack(synth.base_flow(*n, bc, 110 + q))).cuda())
        for r in range(2):  # two vectors per grid: ordered on its branch
            x = torch.from_numpy(synth.krylov_input(*n, 120 + 2 * q + r)[0]).cuda()
            y = g.empty(4)
            plan.add(g, x, y)
            xs.append(x)
            ys.append(y)
            refs.append((g, x))
        grids.append(g)
    for _ in range(2):  # capture, then replay
        for y in ys:
            y.fill_(float("nan"))
        plan.launch()
        torch.cuda.synchronize()
        for y, (g, x) in zip(ys, refs):
            assert torch.equal(y, g.krylov_vector(x))
    plan.close()


def test_bounded_wait_expiry_is_reported_and_grid_stays_usable():
    """Failure detection without a GPU fault: a contraction whose barriers never complete gives
    up after its bounded waits and reports through the device error flag; afterwards the same
    grid still computes correct Krylov vectors."""
    from paper_1905_11601_gb300 import kv
    n = (24, 20, 18)
    base = torch.from_numpy(np.stack(synth.base_flow(*n, synth.CC, 131))).cuda()
    x = torch.from_numpy(synth.krylov_input(*n, 132)[0]).cuda()
    g64 = kv.Grid(*n, gr=2e6)
    g64.set_base_flow(base)
    ref = g64.krylov_vector(x)
    g = kv.Grid(*n, gr=2e6, precision=kv.KV_PREC_MIXED)
    g.set_base_flow(base)
    assert g.selftest_wait_timeout() != 0
    y, st = g.krylov_vector(x, stats=True)
    assert st.device_error == 0
    err = (torch.linalg.vector_norm(y - ref) / torch.linalg.vector_norm(ref)).item()
    assert err < 1e-9


def test_host_stream_matches_single_host_calls():
    """The streamed host-buffer entry point (copies overlapping the evaluations, two staging
    slots) gives the same vectors as one kv_krylov_vector_host call per vector, for an odd count
    that cycles both slots, in both precisions."""
    from paper_1905_11601_gb300 import kv
    n = (24, 20, 18)
    base = np.stack(synth.base_flow(*n, synth.CC, 51))
    X = np.stack([synth.krylov_input(*n, 52 + i)[0] for i in range(5)])
    for prec in (kv.KV_PREC_FP64, kv.KV_PREC_MIXED):
        g = kv.Grid(*n, gr=2e6, pr=0.71, precision=prec)
        g.set_base_flow(torch.from_numpy(base).cuda())
        Xh = torch.from_numpy(X.reshape(5, -1).copy()).pin_memory()
        Yh = torch.zeros_like(Xh).pin_memory()
        g.krylov_vector_host_stream(Xh, Yh)
        for i in range(5):
            y1 = torch.zeros(Xh.shape[1], dtype=torch.float64).pin_memory()
            g.krylov_vector_host(Xh[i].contiguous(), y1)
            assert torch.equal(Yh[i], y1), (prec, i)
        g.krylov_vector_host_stream(Xh[:0], Yh[:0])  # nb = 0 does nothing


@pytest.mark.parametrize("n,bc,tproj,count", [((70, 65, 67), synth.CC, 0, 3), ((33, 18, 20), synth.AA, 1, 18)])
def test_mixed_blocks_equal_single_calls(n, bc, tproj, count):
    """Mixed-precision batches go through blocks of up to 16 vectors whose tensor-core
    contractions are one launch per axis for the whole block. Each vector's tiles do the same
    arithmetic as a single evaluation, so the results equal single calls bit for bit: on a grid
    whose cell count is not a multiple of 4 (the contraction's epilogue then takes its scalar
    stores) and for 18 vectors (a block of 16 and one of 2), insulated walls, oblique reading."""
    from paper_1905_11601_gb300 import kv
    g = kv.Grid(*n, bc=bc, gr=3e6, tproj=tproj, precision=kv.KV_PREC_MIXED)
    g.set_base_flow(torch.from_numpy(np.stack(synth.base_flow(*n, bc, 141))).cuda())
    X = torch.from_numpy(synth.krylov_input(*n, 142, count=count)).cuda()
    ref = torch.stack([g.krylov_vector(X[b].contiguous()) for b in range(count)])
    g.guard(reset=True)
    Y = g.krylov_vector_batch(X)
    torch.cuda.synchronize()
    assert torch.equal(Y, ref)
    gd = g.guard()
    assert gd["checks"] == count and gd["failed"] == 0 and gd["nonfinite"] == 0, gd
