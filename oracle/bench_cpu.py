"""Times the FP64 CPU oracle on a workload (test infrastructure: the benchmark's CPU
baseline). Prints one JSON line: Krylov-vector evaluations per second on the host cores.

    python -m oracle.bench_cpu --workload cube256_cc --evals 1 [--warmup 0] [--best-of 1] [--stretch 0.12]
    python -m oracle.bench_cpu --workload cube256_cc --arnoldi 5 --evals 8 [--restart 20]
    python -m oracle.bench_cpu --newton-cycle 20
    python -m oracle.bench_cpu --plan   # 100^3, 128^3, 256^3 on all cores and on 1 core, best of 5

With --best-of B the figure is the fastest of B timed evaluations (after the warm-up); cores is
the number of OpenMP threads the oracle ran with (OMP_NUM_THREADS, else all host cores).
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
    print(json.dumps({"value": info["matvecs"] / dt, "unit": "Krylov-vector evals/s inside the solves",
                      "seconds": dt, "matvecs": info["matvecs"], "cores": threads(),
                      "sample": f"one GMRES({m}) cycle of the first Newton correction at 64^3, CC, Gr = 1e4"}))


def host_info():
    """nproc and the lscpu model line of the host, for the record."""
    import subprocess
    info = {"nproc": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() in ("Model name", "Architecture", "CPU(s)", "Socket(s)", "Core(s) per socket"):
                info[k.strip()] = v.strip()
    except Exception:
        pass
    return info


def threads():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def arnoldi(w, j0, steps, restart):
    """Oracle Arnoldi steps (Krylov vector + classical Gram-Schmidt twice + normalisation) at the
    basis sizes the GPU benchmark times: the basis V_0..V_j0 is made orthonormal first (numpy,
    untimed), then `steps` steps from j = j0 are timed, restarting from the last vector after
    `restart` vectors as the benchmark does."""
    base, x = synth.workload_arrays(w)
    base = np.stack(base)
    o = Oracle(w.nx, w.ny, w.nz, bc=w.bc, gr=w.gr, pr=w.pr)
    V = np.zeros((restart + 1, 4) + o.shape)
    v = o.project_input(x[0])
    V[0] = v / np.linalg.norm(v)
    rng = np.random.default_rng(w.seed + 7)
    for q in range(1, j0 + 1):
        r = rng.standard_normal(V[0].shape)
        for p in range(q):
            r -= np.vdot(V[p], r) * V[p]
        V[q] = r / np.linalg.norm(r)
    o.krylov_vector(base, V[0])  # warm-up (untimed)
    j, nq = j0, []
    t0 = time.perf_counter()
    for _ in range(steps):
        if j == restart:
            V[0] = V[restart]
            j = 0
        o.arnoldi_step(base, V, j)
        nq.append(j + 1)
        j += 1
    dt = time.perf_counter() - t0
    return {"value": steps / dt, "unit": "Krylov-vector evals/s", "seconds": dt, "steps": steps, "nq": nq,
            "cores": threads(), "workload": w.name, "host": host_info()}


def plan():
    """The CPU baseline plan: 100^3, 128^3 and 256^3 (the benchmark's CC workloads), all cores and
    one core, best of 5 after one warm-up evaluation (256^3 on one core: best of 2)."""
    import subprocess
    rows = []
    for wl in ("cube100_cc", "cube128_aa", "cube256_cc"):
        for one in (False, True):
            env = dict(os.environ)
            if one:
                env["OMP_NUM_THREADS"] = "1"
            best = 2 if (one and wl == "cube256_cc") else 5
            cmd = [sys.executable, "-m", "oracle.bench_cpu", "--workload", wl, "--evals", "1", "--warmup", "1",
                   "--best-of", str(best)]
            r = subprocess.run(cmd, cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))), env=env,
                               capture_output=True, text=True)
            rows.append(json.loads(r.stdout.strip().splitlines()[-1]))
    print(json.dumps({"plan": rows, "host": host_info()}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="cube256_cc")
    ap.add_argument("--evals", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=0)
    ap.add_argument("--newton-cycle", type=int, default=0, help="time one GMRES(m) cycle of the Newton line instead")
    ap.add_argument("--stretch", type=float, default=0.0, help="grid stretching parameter of Eq (22)")
    ap.add_argument("--adv", type=int, default=0, help="advection scheme: 0 central, 1 first-order upwind")
    ap.add_argument("--best-of", type=int, default=1, help="report the fastest of this many timed repetitions")
    ap.add_argument("--arnoldi", type=int, default=-1, help="time Arnoldi steps from this basis index instead")
    ap.add_argument("--restart", type=int, default=20)
    ap.add_argument("--plan", action="store_true", help="run the whole CPU baseline plan")
    a = ap.parse_args()
    if a.newton_cycle:
        newton_cycle(a.newton_cycle)
        return
    if a.plan:
        plan()
        return
    w = synth.WORKLOADS[a.workload]
    if a.arnoldi >= 0:
        print(json.dumps(arnoldi(w, a.arnoldi, a.evals, a.restart)))
        return
    base, x = synth.workload_arrays(w)
    base = np.stack(base)
    t0 = time.perf_counter()
    o = Oracle(w.nx, w.ny, w.nz, bc=w.bc, gr=w.gr, pr=w.pr, stretch=a.stretch, adv=a.adv)
    setup = time.perf_counter() - t0
    for _ in range(a.warmup):
        o.krylov_vector(base, x[0])
    times = []
    for _ in range(max(1, a.best_of)):
        t0 = time.perf_counter()
        for _ in range(a.evals):
            o.krylov_vector(base, x[0])
        times.append(time.perf_counter() - t0)
    dt = min(times)
    print(json.dumps({"value": a.evals / dt, "unit": "Krylov-vector evals/s", "seconds": dt, "evals": a.evals,
                      "best_of": len(times), "all_seconds": times, "warmup": a.warmup, "cores": threads(),
                      "workload": a.workload, "stretch": a.stretch, "adv": a.adv, "setup_seconds": setup, "host": host_info()}))


if __name__ == "__main__":
    main()
