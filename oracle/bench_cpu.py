"""Times the FP64 CPU oracle on a workload (test infrastructure: the benchmark's CPU
baseline). Prints one JSON line: Krylov-vector evaluations per second on the host cores.

    python -m oracle.bench_cpu --workload cube256_cc --evals 1 [--warmup 0] [--stretch 0.12]
    python -m oracle.bench_cpu --newton-cycle 20
"""
import argparse
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from oracle import Oracle  # noqa: E402
from paper_1905_11601_gb300 import synth  # noqa: E402


def newton_cycle(m):
    """One GMRES(m) cycle of the first Newton correction at 64^3 (CC, Gr = 1e4, the synthetic base
    flow of the benchmark's Newton line): the oracle's Krylov vectors per second inside the
    solver."""
    from oracle.solvers import gmres

    n = 64
    S = np.stack(synth.base_flow(n, n, n, synth.CC, 11900))
    o = Oracle(n, n, n, bc=synth.CC, gr=1e4, pr=0.71)
    F, _ = o.newton_residual(S)
    t0 = time.perf_counter()
    _, info = gmres(lambda v: o.krylov_vector(S, v), F, np.zeros_like(F), m, 1, 0.0)
    dt = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    print(json.dumps({"value": info["matvecs"] / dt, "unit": "Krylov-vector evals/s inside the solves",
                      "seconds": dt, "matvecs": info["matvecs"], "cores": threads,
                      "sample": f"one GMRES({m}) cycle of the first Newton correction at 64^3, CC, Gr = 1e4"}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="cube256_cc")
    ap.add_argument("--evals", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=0)
    ap.add_argument("--newton-cycle", type=int, default=0, help="time one GMRES(m) cycle of the Newton line instead")
    ap.add_argument("--stretch", type=float, default=0.0, help="grid stretching parameter of Eq (22)")
    a = ap.parse_args()
    if a.newton_cycle:
        newton_cycle(a.newton_cycle)
        return
    w = synth.WORKLOADS[a.workload]
    base, x = synth.workload_arrays(w)
    base = np.stack(base)
    t0 = time.perf_counter()
    o = Oracle(w.nx, w.ny, w.nz, bc=w.bc, gr=w.gr, pr=w.pr, stretch=a.stretch)
    setup = time.perf_counter() - t0
    for _ in range(a.warmup):
        o.krylov_vector(base, x[0])
    t0 = time.perf_counter()
    for _ in range(a.evals):
        o.krylov_vector(base, x[0])
    dt = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    print(json.dumps({"value": a.evals / dt, "unit": "Krylov-vector evals/s", "seconds": dt, "evals": a.evals,
                      "cores": threads, "workload": a.workload, "stretch": a.stretch, "setup_seconds": setup}))


if __name__ == "__main__":
    main()
