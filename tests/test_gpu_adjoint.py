"""GPU parity of the transpose of the Krylov map and of the base-flow sensitivities (the adjoint
form): against the oracle's transpose (formed entry by entry from the definition of J), the
dot-product test, and central finite differences of the Rayleigh quotient through the
torch.autograd.Function."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1905_11601_gb300 import synth
from tests.oracle_helpers import project_output_side

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
RTOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_11601_gb300 import build
    build.build()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def grid(n, bc, gr, base, precision=0):
    from paper_1905_11601_gb300 import kv
    g = kv.Grid(*n, bc=bc, gr=gr, pr=0.71, precision=precision)
    g.set_base_flow(torch.from_numpy(base).cuda())
    return g


CASES = [((24, 24, 24), synth.CC, 2.5e6), ((17, 12, 9), synth.AA, 3e6), ((5, 4, 6), synth.CC, 1e6)]


@pytest.mark.parametrize("n,bc,gr", CASES)
def test_adjoint_matches_oracle_transpose(n, bc, gr):
    base = np.stack(synth.base_flow(*n, bc, 91))
    y = synth.krylov_input(*n, 92)[0]
    g = grid(n, bc, gr, base)
    z = g.krylov_vector_adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    z_ref = Oracle(*n, bc=bc, gr=gr).krylov_adjoint(base, y)
    assert rel(z, z_ref) < RTOL


@pytest.mark.parametrize("n,bc,gr", CASES)
def test_base_flow_gradient_matches_oracle(n, bc, gr):
    base = np.stack(synth.base_flow(*n, bc, 93))
    x = synth.krylov_input(*n, 94, 2)
    g = grid(n, bc, gr, base)
    gt, dgr = g.base_flow_gradient(torch.from_numpy(x[0]).cuda(), torch.from_numpy(x[1]).cuda())
    o = Oracle(*n, bc=bc, gr=gr)
    xp, yh = o.project_input(x[0]), project_output_side(o, x[1])
    gb = o.grad_base(xp, yh)
    gt = gt.cpu().numpy()
    assert rel(gt[3], gb[3]) < RTOL
    for c in range(3):  # the base velocity components
        assert rel(gt[c], gb[c]) < RTOL, c
    assert abs(dgr - o.grad_gr(xp, yh)) < RTOL * abs(dgr) * 10


@pytest.mark.parametrize("precision,tol", [(0, 1e-13), (1, 1e-9)])
def test_dot_product_at_64(precision, tol):
    n = (64, 64, 64)
    base = np.stack(synth.base_flow(*n, synth.CC, 95))
    g = grid(n, synth.CC, 2e6, base, precision)
    x = torch.from_numpy(synth.krylov_input(*n, 96, 2)).cuda()
    Ax = g.krylov_vector(x[0].contiguous())
    ATy = g.krylov_vector_adjoint(x[1].contiguous())
    lhs, rhs = torch.vdot(x[1].flatten(), Ax.flatten()).item(), torch.vdot(ATy.flatten(), x[0].flatten()).item()
    scale = (torch.linalg.vector_norm(x[1]) * torch.linalg.vector_norm(Ax)).item()
    assert abs(lhs - rhs) < tol * scale


def test_rayleigh_quotient_gradient_autograd_at_160():
    """The adjoint workload: R = <y, A(Theta) x> / <y, x> on the 160^3 grid (Gr = 2.5e6, CC);
    dR/dTheta from the autograd backward pass against a central difference with h = 1e-6 (R is
    affine in Theta, so the difference is exact up to rounding)."""
    from paper_1905_11601_gb300 import kv
    from paper_1905_11601_gb300.autograd import krylov_map
    w = synth.WORKLOADS["cube160_cc"]
    n = (w.nx, w.ny, w.nz)
    base = torch.from_numpy(np.stack(synth.base_flow(*n, w.bc, w.seed))).cuda()
    xs = torch.from_numpy(synth.krylov_input(*n, w.seed, 2)).cuda()
    x, y = xs[0].contiguous(), xs[1].contiguous()
    g = kv.Grid(*n, bc=w.bc, gr=w.gr, pr=w.pr)
    vel = base[:3].contiguous()
    theta = base[3].clone().requires_grad_(True)
    yx = torch.vdot(y.flatten(), x.flatten())
    R = torch.vdot(y.flatten(), krylov_map(x, theta, g, vel).flatten()) / yx
    R.backward()
    grad = theta.grad
    d = torch.from_numpy(np.random.default_rng(97).standard_normal(tuple(theta.shape))).cuda()
    h = 1e-6
    with torch.no_grad():
        Rp = torch.vdot(y.flatten(), krylov_map(x, base[3] + h * d, g, vel).flatten()) / yx
        Rm = torch.vdot(y.flatten(), krylov_map(x, base[3] - h * d, g, vel).flatten()) / yx
    fd = ((Rp - Rm) / (2 * h)).item()
    an = torch.vdot(grad.flatten(), d.flatten()).item()
    assert abs(fd - an) < 1e-6 * abs(an)
    # the base-velocity gradient along a random direction (A is affine in U as well)
    velr = vel.clone().requires_grad_(True)
    R3 = torch.vdot(y.flatten(), krylov_map(x, base[3], g, velr).flatten()) / yx
    R3.backward()
    du = torch.from_numpy(np.random.default_rng(98).standard_normal(tuple(vel.shape))).cuda()
    with torch.no_grad():
        Rp = torch.vdot(y.flatten(), krylov_map(x, base[3], g, (vel + h * du).contiguous()).flatten()) / yx
        Rm = torch.vdot(y.flatten(), krylov_map(x, base[3], g, (vel - h * du).contiguous()).flatten()) / yx
    fd = ((Rp - Rm) / (2 * h)).item()
    an = torch.vdot(velr.grad.flatten(), du.flatten()).item()
    assert abs(fd - an) < 1e-6 * abs(an)
    # the x gradient of R is A^T y / <y, x> (through the same function)
    xr = x.clone().requires_grad_(True)
    R2 = torch.vdot(y.flatten(), krylov_map(xr, base[3], g, vel).flatten()) / yx
    R2.backward()
    z = g.krylov_vector_adjoint(y) / yx
    assert (torch.linalg.vector_norm(xr.grad - z) / torch.linalg.vector_norm(z)).item() < 1e-14
