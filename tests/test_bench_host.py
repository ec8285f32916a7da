"""Host logic of bench.py's roofline objects (no GPU): the algorithmic bytes of the delayed
Gram-Schmidt sweeps, the per-run bytes of each run's last vector, and the traffic entries that
follow the kernel sources."""
import json
import os

import pytest

import bench
from paper_1905_11601_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def phases(ms):
    return {k: {"ms": v, "timed": 1, "launches": 1} for k, v in ms.items()}


def test_update_sweep_bytes_and_kernel():
    w = synth.WORKLOADS["cube256_cc"]
    L = 4 * 258 ** 3
    nqs = list(range(4, 14))  # ten steps, basis sizes 4..13, one run
    r = bench.roofline(phases({"gs_update": 10.0, "gs_dots": 9.0}), w, "mixed", 10, nqs)
    assert r["kernel"].startswith("k_update2")
    byts = 8.0 * L * sum(nq + 3 for nq in nqs)
    assert r["achieved"] == pytest.approx(byts / 10e-3 / 1e9)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"


def test_inner_product_sweep_bytes():
    w = synth.WORKLOADS["cube256_cc"]
    L = 4 * 258 ** 3
    nqs = [4, 5, 6]
    r = bench.roofline(phases({"gs_dots": 3.0}), w, "mixed", 3, nqs)
    assert r["kernel"].startswith("k_dots2")
    assert r["achieved"] == pytest.approx(8.0 * L * sum(nq + 1 for nq in nqs) / 3e-3 / 1e9)


def test_last_vector_sweeps_once_per_run():
    """Two runs (a restart after basis size 20): the last vector's sweeps are counted once per
    run, at each run's final basis size."""
    w = synth.WORKLOADS["cube256_cc"]
    L = 4 * 258 ** 3
    nqs = [18, 19, 20, 1, 2]
    r = bench.roofline(phases({"arnoldi": 5.0}), w, "mixed", 5, nqs)
    byts = 8.0 * L * ((20 + 1) + (20 + 2) + (2 + 1) + (2 + 2))
    assert r["achieved"] == pytest.approx(byts / 5e-3 / 1e9)


def test_traffic_entries_follow_their_sources():
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for kern, e in d.items():
        if kern.startswith("_"):
            continue
        src = os.path.join(ROOT, "paper_1905_11601_gb300", "csrc", e["source"])
        assert os.path.exists(src), kern
        got = bench.traffic_for(kern, 1.0)
        if bench.source_sha(src) == e["source_sha"]:
            assert got == pytest.approx(e["bytes_per_unit"]), kern
        else:
            assert got is None, kern
