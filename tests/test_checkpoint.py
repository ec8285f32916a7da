"""Arnoldi checkpoint / resume: the basis, the Hessenberg matrix and the step count survive a
save and a load bit for bit (CPU tensors; no GPU needed)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_arnoldi_state_round_trip(tmp_path):
    from paper_1905_11601_gb300.arnoldi import load_state, save_state
    rng = np.random.default_rng(5)
    V = torch.from_numpy(rng.standard_normal((6, 4, 5, 4, 3)))
    H = rng.standard_normal((6, 5))
    save_state(tmp_path / "ck.pt", V, H, 4)
    V2, H2, j = load_state(tmp_path / "ck.pt", device="cpu")
    assert torch.equal(V, V2) and np.array_equal(H, H2) and j == 4
