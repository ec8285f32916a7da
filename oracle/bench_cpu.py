"""Times the FP64 CPU oracle on a workload (test infrastructure: the benchmark's CPU
baseline). Prints one JSON line: Krylov-vector evaluations per second on the host cores.

    python -m oracle.bench_cpu --workload cube256_cc --evals 1 [--warmup 0]
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="cube256_cc")
    ap.add_argument("--evals", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=0)
    a = ap.parse_args()
    w = synth.WORKLOADS[a.workload]
    base, x = synth.workload_arrays(w)
    base = np.stack(base)
    o = Oracle(w.nx, w.ny, w.nz, bc=w.bc, gr=w.gr, pr=w.pr)
    for _ in range(a.warmup):
        o.krylov_vector(base, x[0])
    t0 = time.perf_counter()
    for _ in range(a.evals):
        o.krylov_vector(base, x[0])
    dt = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    print(json.dumps({"value": a.evals / dt, "unit": "Krylov-vector evals/s", "seconds": dt, "evals": a.evals,
                      "cores": threads, "workload": a.workload}))


if __name__ == "__main__":
    main()
