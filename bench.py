#!/usr/bin/env python
"""Throughput benchmark of the Krylov-vector evaluation (Gelfgat, arXiv 1905.11601, Section 3.1).

One step = one Arnoldi step on the 256^3 grid: the Krylov vector y = (Pi_v (+) P_T) J P_BC x
(linearised operator stencil, divergence, TPF Poisson solve, velocity correction and temperature
projection) followed by classical Gram-Schmidt (twice) against the current basis and the
normalisation; the basis is restarted every --restart vectors. The headline value is the
mixed-precision path (tensor-core Poisson contractions refined to FP64 accuracy); the plain FP64
path is timed on the same workload and reported beside it, with the mixed result's relative
error against it. Inputs are seeded synthetic base
flows and vectors (no dataset), resident in HBM before the timed region; every vector (551 MB)
is larger than L2, so no L2 flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 (launched by torch.distributed.run) every rank runs an independent replica of the
workload on its own GPU (the method needs no exchange between independent problems); the
value is the whole-job rate, the time the maximum over ranks. Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Krylov-vector evals/s at 256^3: mixed vs FP64 plain at 1e-9 rel err; roofline %"
UNIT = "Krylov-vector evals/s"
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 rate (an FMA-loop probe measured 1.20)
FP64_PEAK_SRC = "nominal GB300 FP64 rate (FMA-loop probe on this pool: 1.20 TFLOP/s)"
# The assembled Jacobian J has 60 nonzeros per cell: 15 per velocity face (7 own-field points, 4 + 4
# cross-component points), 13 per temperature cell (7 + 2 + 2 + 2) and 2 for the buoyancy term.
STENCIL_FLOPS_PER_CELL = 2 * 60


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="cube256_cc")
    ap.add_argument("--restart", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the 16-vector block and the 12-grid plan measurements")
    ap.add_argument("--single", choices=["fp64", "mixed", "mixed-arnoldi", "mixed-arnoldi-run", "mixed-newton"],
                    default=None,
                    help="profiling case: two untimed Krylov-vector evaluations (or 8 Arnoldi steps, step by step "
                         "or as one kv_arnoldi_run, or two Newton corrections at 64^3 with one GMRES(30) cycle "
                         "each), no JSON line")
    ap.add_argument("--operator", default=None, metavar="VARIANT,PLANES",
                    help="with --single: pin the mixed path's operator (kv_set_tuning), e.g. 2,16 for the "
                         "fixed-point march with 16 planes per block, 1,32 for the double-float march")
    ap.add_argument("--advection", choices=["central", "upwind"], default="central",
                    help="with --single: the advection scheme of the operator (KV_ADV_*)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm, src = 6783.0, "measured copy bandwidth of this pool's GB300 (6783 GB/s)"
    try:
        d = json.load(open(path))
        for key in ("hbm_gbs", "hbm_GBs", "hbm"):
            if key in d and isinstance(d[key], (int, float)):
                hbm, src = float(d[key]), "MEASURED_PEAKS.json"
                break
    except Exception:
        pass
    return hbm, src


def workload_desc(w, restart, precision="fp64"):
    bc = "CC" if w.bc == 0 else "AA"
    return {"workload": f"{w.name}: {w.nx}x{w.ny}x{w.nz} MAC grid, {bc} spanwise walls, Gr={w.gr:g}, "
                        f"Pr={w.pr:g}, Arnoldi step (Krylov vector + CGS2), restart {restart}, {precision}",
            "grid": [w.nx, w.ny, w.nz], "spanwise_bc": bc, "gr": w.gr, "pr": w.pr, "restart": restart,
            "precision": precision,
            "l2": "inputs larger than L2 (one packed FP64 vector is "
                  f"{4 * (w.nx + 2) * (w.ny + 2) * (w.nz + 2) * 8 / 1e6:.0f} MB), no flush"}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.QUERY}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().splitlines() if r.strip()]
        self.f.close()
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [c.strip() for c in r]
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def bf16_peak():
    """Dense BF16 tensor peak (TFLOP/s) for a kernel timed inside a long step: the sustained figure."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        for key in ("bf16_tflops_sustained", "bf16_sustained_tflops"):
            if key in d and isinstance(d[key], (int, float)):
                return float(d[key]), "MEASURED_PEAKS.json (sustained)"
    except Exception:
        pass
    return 1730.0, "measured sustained cuBLAS BF16 on this pool's GB300 (1730 TFLOP/s)"


def source_sha(path):
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def traffic_for(kernel, units=None):
    """DRAM bytes per launch of a kernel from a committed ncu summary (profiles/traffic.json), if
    the kernel's source is unchanged since the capture. Entries either give bytes per launch of
    this workload, or bytes per unit measured on a smaller case (scaled by `units`)."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
        src = os.path.join(ROOT, "paper_1905_11601_gb300", "csrc", d["source"])
        if source_sha(src) != d["source_sha"]:
            return None
        if "bytes_per_unit" in d:
            return None if units is None else d["bytes_per_unit"] * units
        return d["bytes_per_launch"]
    except Exception:
        return None


DTYPE_MIXED = "mixed: bf16 tensor-core slices (fp32 accumulate) + fp32-pair double-float + f64"


def cpu_baseline(workload, evals, warmup, timeout=900, best_of=1, one_core=False, extra=()):
    cmd = [sys.executable, "-m", "oracle.bench_cpu", "--workload", workload, "--evals", str(evals),
           "--warmup", str(warmup), "--best-of", str(best_of)] + list(extra)
    env = dict(os.environ)
    if one_core:
        env["OMP_NUM_THREADS"] = "1"
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=timeout, env=env)
    if r.returncode != 0:
        raise RuntimeError(f"oracle baseline failed: {r.stderr[-2000:]}")
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1905_11601_gb300 import synth
    w = synth.WORKLOADS[args.workload]
    # each oracle step is one full Arnoldi step of the same workload on the host cores (the
    # Krylov vector, classical Gram-Schmidt twice and the normalisation), at the basis sizes the
    # GPU arm times (the first timed step follows `warmup` steps from a one-vector basis); the
    # counts are capped so the run stays within a few minutes
    steps = max(1, min(args.steps, 8))
    j0 = args.warmup % args.restart
    r = cpu_baseline(args.workload, steps, 0, extra=["--arnoldi", str(j0), "--restart", str(args.restart)])
    warm = 1
    sample = (f"{steps} timed FP64 oracle Arnoldi steps of {w.name} (Krylov vector + CGS2 + normalisation) at "
              f"basis sizes {r['nq']}, after one untimed Krylov-vector evaluation, on {r['cores']} host threads "
              f"(nproc {r['host'].get('nproc')}, {r['host'].get('Model name', 'host CPU')})")
    out = {"impl": "reference", "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": args.gpus,
           "steps": steps, "warmup": warm, "ms_per_step": 1000.0 / r["value"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_desc(w, args.restart, "mixed"),
           "cpu_baseline": {"value": r["value"], "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": r["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def max_over_ranks(x, dist, device="cuda"):
    """Maximum of a per-rank scalar over all ranks (the job's time is the slowest replica's)."""
    if not dist:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds_max):
    """Units processed by all replicas divided by the slowest replica's time (weak scaling)."""
    return world * units_per_rank / seconds_max


def arnoldi_run(g, V, m, steps, warmup, dist, clocks_index=None, delayed=True):
    """Times `steps` Arnoldi steps (after `warmup`) on the current stream; restart every m.
    delayed: the steps between restarts as one kv_arnoldi_run call (delayed classical
    Gram-Schmidt, one synchronisation per call); else one kv_arnoldi_step call per step."""
    import numpy as np
    import torch

    state = {"j": 0, "nq": [], "runs": 0}
    H = np.zeros((m + 1, m))

    def run_steps(n):
        left = n
        while left > 0:
            j = state["j"]
            if j == m:  # restart the basis from the last vector
                V[0].copy_(V[m])
                j = 0
            k = min(left, m - j)
            if delayed:
                Hn = g.arnoldi_run(V, j, k, H)
                H[: j + k + 1, : j + k] = Hn
            else:
                for jj in range(j, j + k):
                    H[: jj + 2, jj] = g.arnoldi_step(V, jj)
            state["nq"].extend(range(j + 1, j + k + 1))
            state["runs"] += 1
            state["j"] = j + k
            left -= k

    run_steps(warmup)
    state["nq"].clear()
    state["runs"] = 0
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(clocks_index) if clocks_index is not None else None
    j0 = state["j"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run_steps(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    ms = max_over_ranks(e0.elapsed_time(e1), dist)
    # phase breakdown from a second pass over the same basis sizes with the library's per-phase
    # CUDA events on (kept out of the timed region above)
    nq_timed = list(state["nq"])
    runs = state["runs"]
    state["nq"].clear()
    state["j"] = j0
    g.profile_enable(True)
    run_steps(steps)
    torch.cuda.synchronize()
    prof = g.profile()
    counts = g.arnoldi_counts()  # (fused steps, of them with the second update) of this pass
    g.profile_enable(False)
    phases = {k: {"ms": v[0], "timed": v[1], "launches": v[2]} for k, v in prof.items()}
    total = sum(p["ms"] for p in phases.values())
    for p in phases.values():
        p["share"] = p["ms"] / total if total else None
    assert state["nq"] == nq_timed
    return ms, phases, clk, nq_timed, counts, runs


def roofline(phases, w, precision, steps, nqs=(), tuning=None):
    """Roofline of the dominant kernel (largest share of the timed region)."""
    n3 = w.nx * w.ny * w.nz
    L = 4 * (w.nx + 2) * (w.ny + 2) * (w.nz + 2)
    dom = max(phases, key=lambda k: phases[k]["ms"])
    hbm_peak, hbm_src = measured_peaks()
    avg_ms = phases[dom]["ms"] / max(phases[dom]["timed"], 1)
    if dom == "tpd" and precision == "fp64":
        flops = 2.0 * (n3 * w.nx + n3 * w.ny + n3 * w.nz) / 3.0
        ach = flops / (avg_ms / 1e3) / 1e12
        return {"kernel": "k_gemm_axis (FP64 per-axis TPF contraction)", "bound": "alu", "achieved": ach,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS,
                "traffic": traffic_for("k_gemm_axis"), "peak_source": FP64_PEAK_SRC,
                "algorithmic": f"2 n^4 = {flops:.4g} flop per launch"}
    if dom == "tpd":
        flops = 6 * 2.0 * (n3 * w.nx + n3 * w.ny + n3 * w.nz) / 3.0
        peak, src = bf16_peak()
        ach = flops / (avg_ms / 1e3) / 1e12
        return {"kernel": "k_umma_axis (tcgen05 BF16-slice TPF contraction)", "bound": "tensor", "achieved": ach,
                "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": traffic_for("k_umma_axis"),
                "peak_source": src, "algorithmic": f"6 slice products x 2 n^4 = {flops:.4g} flop per launch"}
    if dom == "stencil" and precision == "fp64":
        flops = STENCIL_FLOPS_PER_CELL * n3
        ach = flops / (avg_ms / 1e3) / 1e12
        return {"kernel": "k_apply (FP64 assembled linearised operator)", "bound": "alu", "achieved": ach,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS,
                "traffic": traffic_for("k_apply"), "peak_source": FP64_PEAK_SRC,
                "algorithmic": f"{STENCIL_FLOPS_PER_CELL} flop per cell (2 per Jacobian nonzero) = {flops:.4g} per launch"}
    if dom == "stencil":
        # J x: read x (4 fields) and the base state (4), write v* and T* (4): 12 x 8 B per cell
        byts = 12 * 8.0 * n3
        ach = byts / (avg_ms / 1e3) / 1e9
        variant = tuning.get("df_variant") if tuning else None
        points = (w.nx + 2) * (w.ny + 2) * (w.nz + 2)
        if variant == 2:
            tf = [traffic_for(k, points) for k in ("k_fx_prepass", "k_apply_fx_march")]
            return {"kernel": "k_fx_prepass + k_apply_fx_march (fixed-point operator from the base state)",
                    "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                    "traffic": None if None in tf else sum(tf), "peak_source": hbm_src,
                    "algorithmic": f"12 fields x 8 B per cell = {byts:.4g} B per evaluation (read x and the base "
                                   f"state, write v* and T*); traffic: measured DRAM bytes of both kernels per "
                                   f"evaluation (the pre-pass reads x once more for its largest magnitude)"}
        march = variant == 1
        name = ("k_zero_boundary + k_apply_df_march (double-float operator, 2.5D march)" if march
                else "k_split_input + k_apply_df (double-float operator)")
        return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "traffic": traffic_for("k_apply_df_march", points) if march else None,
                "peak_source": hbm_src,
                "algorithmic": f"12 fields x 8 B per cell = {byts:.4g} B per evaluation; the assembled form reads "
                               f"25 coefficient pairs per cell instead of the 4 base fields (traffic: measured "
                               f"DRAM bytes per launch, about 2.7x the algorithmic bytes), to keep the FP64-accurate "
                               f"operator off GB300's FP64 pipe"}
    if dom in ("gs_update", "gs_dots", "arnoldi") and nqs:
        # The delayed classical Gram-Schmidt (kv_arnoldi_run): per step (basis size nq after it),
        # the inner-product sweep streams nq + 1 vectors (the nq - 1 final ones, the provisional
        # vector and its image) and the update sweep reads nq + 1 and writes 2; per run, the last
        # vector's two sweeps stream (J + 1) + (J + 2) vectors, J the run's final basis size.
        ends = [nq for i, nq in enumerate(nqs) if i + 1 == len(nqs) or nqs[i + 1] <= nq]
        if dom == "arnoldi":
            units = L * sum((J + 1) + (J + 2) for J in ends) / len(nqs)
            byts = 8.0 * units * len(nqs)
            ach = byts / (phases[dom]["ms"] / 1e3) / 1e9
            return {"kernel": "k_dcgs_coef + the last vector's sweeps (k_dots_df, k_update2)", "bound": "hbm",
                    "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak, "traffic": None,
                    "peak_source": hbm_src,
                    "algorithmic": "(J + 1) + (J + 2) vectors x 8 B per entry per run, J the run's basis size"}
        per = [(nq + 1) if dom == "gs_dots" else (nq + 3) for nq in nqs]
        units = L * sum(per) / len(per)
        kern = {"gs_dots": "k_dots2", "gs_update": "k_update2"}[dom]
        if precision == "fp64":
            # per entry and step: 2 (nq - 1) + 3 multiply-adds in either sweep, FP64
            flops = 2.0 * L * sum(2 * nq + 1 for nq in nqs)
            ach = flops / (phases[dom]["ms"] / 1e3) / 1e12
            return {"kernel": kern + " (FP64 Gram-Schmidt sweep)", "bound": "alu", "achieved": ach,
                    "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS,
                    "traffic": traffic_for(kern, units), "peak_source": FP64_PEAK_SRC,
                    "algorithmic": f"2 x (2 nq + 1) flop per vector entry per launch, nq = basis size, "
                                   f"mean nq {sum(nqs) / len(nqs):.1f}"}
        byts = 8.0 * L * sum(per)
        ach = byts / (phases[dom]["ms"] / 1e3) / 1e9
        name = {"gs_dots": "k_dots2 (inner products of the basis with the provisional vector and its image, "
                           "double-float and FP64)",
                "gs_update": "k_update2 (final vector and next provisional vector, double-float and FP64)"}[dom]
        return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "traffic": traffic_for(kern, units), "peak_source": hbm_src,
                "algorithmic": f"(nq + 1) or (nq + 3) vectors x 8 B per entry per launch, "
                               f"mean nq {sum(nqs) / len(nqs):.1f}"}
    # b = D v*: read 3 fields, write 1; v = v* - G phi: read v* (3) and phi (1), write 3; residual:
    # read b and phi, write three BF16 slices
    byts = {"divergence": 4 * 8.0 * n3, "correct": 7 * 8.0 * n3, "refine": (2 * 8.0 + 6.0) * n3}.get(dom)
    ach = byts / (avg_ms / 1e3) / 1e9 if byts else None
    return {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
            "frac": ach / hbm_peak if ach else None, "traffic": None, "peak_source": hbm_src}


def timed(fn, reps, warm=1):
    """Seconds per call of fn on the current stream (CUDA events)."""
    import torch
    for _ in range(warm):
        fn()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / reps


def extras(base_np, x_np, w, kv, synth):
    """The batched forms: a block of 16 right-hand sides at 256^3 replayed from one CUDA graph,
    and a plan of 12 grids {100^3 x4, 128^3 x4, 200^3 x2, 256^3 x2} (Gr in [1e6, 4e6], both
    spanwise boundary types) evaluated by one graph launch; a 100-step Arnoldi run at 256^3;
    Newton's method for a steady state at 64^3 (these mixed precision); and one Krylov vector of
    the bench workload on the grid stretched by Eq (22), FP64 and mixed precision; and one Krylov
    vector of the bench workload with first-order upwind advection, FP64 and mixed precision; and
    10 Arnoldi steps by kv_arnoldi_run beside the same steps by kv_arnoldi_step."""
    import numpy as np
    import torch

    out = {}
    g = kv.Grid(w.nx, w.ny, w.nz, bc=w.bc, gr=w.gr, pr=w.pr, precision=kv.KV_PREC_MIXED)
    g.set_base_flow(torch.from_numpy(np.stack(base_np)).cuda())
    X = torch.from_numpy(synth.krylov_input(w.nx, w.ny, w.nz, w.seed + 100, count=16)).cuda()
    Y = torch.empty_like(X)
    t = timed(lambda: g.krylov_vector_batch(X, Y), reps=3)
    out["block16"] = {"workload": f"{w.name}, 16 seeded N(0,1) right-hand sides, one CUDA graph",
                      "value": 16 / t, "unit": UNIT, "ms_per_block": t * 1e3}
    del X, Y, g
    torch.cuda.empty_cache()
    specs = [(100, 0, 1.0e6), (100, 1, 1.6e6), (100, 0, 2.2e6), (100, 1, 2.8e6), (128, 0, 1.4e6), (128, 1, 2.0e6),
             (128, 0, 2.6e6), (128, 1, 3.2e6), (200, 0, 3.4e6), (200, 1, 3.6e6), (256, 0, 3.8e6), (256, 1, 4.0e6)]
    plan = kv.Plan()
    keep = []
    for q, (n, bc, gr) in enumerate(specs):
        gq = kv.Grid(n, n, n, bc=bc, gr=gr, pr=0.71, precision=kv.KV_PREC_MIXED)
        gq.set_base_flow(torch.from_numpy(np.stack(synth.base_flow(n, n, n, bc, 11700 + q))).cuda())
        xq = torch.from_numpy(synth.krylov_input(n, n, n, 11800 + q)[0]).cuda()
        yq = gq.empty(4)
        plan.add(gq, xq, yq)
        keep.append((gq, xq, yq))
    t = timed(plan.launch, reps=3)
    out["plan12"] = {"workload": "12 grids {100^3 x4, 128^3 x4, 200^3 x2, 256^3 x2}, Gr 1e6..4e6, CC and AA, "
                                 "one CUDA graph with a branch per grid",
                     "value": len(specs) / t, "unit": UNIT, "ms_per_launch": t * 1e3}
    plan.close()
    del keep
    torch.cuda.empty_cache()
    # the same 10 Arnoldi steps as the headline's timed ones (basis sizes 4..13 after 3 steps),
    # step by step (kv_arnoldi_step) and as one kv_arnoldi_run (delayed classical Gram-Schmidt:
    # two sweeps over the basis per step and a final one for the run's last vector)
    g = kv.Grid(w.nx, w.ny, w.nz, bc=w.bc, gr=w.gr, pr=w.pr, precision=kv.KV_PREC_MIXED)
    g.set_base_flow(torch.from_numpy(np.stack(base_np)).cuda())
    V = torch.zeros((21, 4) + g.shape, dtype=torch.float64, device="cuda")
    y0 = g.krylov_vector(torch.from_numpy(x_np[0]).cuda())
    V[0] = y0 / torch.linalg.vector_norm(y0)
    del y0
    H = np.zeros((21, 20))
    for j in range(3):
        H[: j + 2, j] = g.arnoldi_step(V, j)
    V0 = V[:4].clone()
    t_step, t_run = [], []
    for _ in range(3):
        V[:4] = V0
        t_step.append(timed(lambda: [g.arnoldi_step(V, j) for j in range(3, 13)], reps=1, warm=0) / 10)
        V[:4] = V0
        t_run.append(timed(lambda: g.arnoldi_run(V, 3, 10, H), reps=1, warm=0) / 10)
    Vm = V[:14].reshape(14, -1)
    orth = (Vm @ Vm.T - torch.eye(14, dtype=torch.float64, device="cuda")).abs().max().item()
    ts, tr = sorted(t_step)[1], sorted(t_run)[1]
    out["arnoldi_stepwise"] = {"workload": f"{w.name}, 10 Arnoldi steps at basis sizes 4..13, mixed precision",
                               "value": 1.0 / ts, "unit": "Arnoldi steps/s", "ms_per_step": ts * 1e3,
                               "delayed_ms_per_step": tr * 1e3, "orthogonality_delayed": orth,
                               "what": "the headline's steps one kv_arnoldi_step call each (classical Gram-Schmidt "
                                       "with the measured second pass, one synchronisation per step) beside one "
                                       "kv_arnoldi_run over the same steps; median of 3"}
    del V, Vm, V0, g
    torch.cuda.empty_cache()
    # a 100-vector Arnoldi run at 256^3 (a 55 GB FP64 basis), mixed precision
    from paper_1905_11601_gb300.arnoldi import ritz
    g = kv.Grid(w.nx, w.ny, w.nz, bc=w.bc, gr=w.gr, pr=w.pr, precision=kv.KV_PREC_MIXED)
    g.set_base_flow(torch.from_numpy(np.stack(base_np)).cuda())
    k = 100
    V = torch.zeros((k + 1, 4) + g.shape, dtype=torch.float64, device="cuda")
    y0 = g.krylov_vector(torch.from_numpy(x_np[0]).cuda())
    V[0] = y0 / torch.linalg.vector_norm(y0)
    del y0
    # step by step (kv_arnoldi_step), then the same 100 steps as one kv_arnoldi_run
    Hs = np.zeros((k + 1, k))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for j in range(k):
        Hs[: j + 2, j] = g.arnoldi_step(V, j)
    torch.cuda.synchronize()
    t_step = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    H = g.arnoldi_run(V, 0, k)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    Vm = V.reshape(k + 1, -1)
    orth = (Vm @ Vm.T - torch.eye(k + 1, dtype=torch.float64, device="cuda")).abs().max().item()
    theta, _, res = ritz(H, 6)
    out["arnoldi100"] = {"workload": f"{w.name}, 100 Arnoldi steps from one vector (basis {V.numel() * 8 / 1e9:.1f} GB), "
                                     "mixed precision, one kv_arnoldi_run (delayed classical Gram-Schmidt)",
                         "value": k / t, "unit": "Arnoldi steps/s", "seconds": t, "orthogonality": orth,
                         "stepwise_value": k / t_step, "stepwise_seconds": t_step,
                         "max_h_difference_to_stepwise": float(np.abs(H - Hs).max() / np.abs(Hs).max()),
                         "rightmost_ritz": [[float(z.real), float(z.imag)] for z in theta],
                         "ritz_residual": [float(r) for r in res]}
    del V, Vm, g
    torch.cuda.empty_cache()
    # Newton's method (Section 2) for a steady state at 64^3 (CC, Gr = 1e4) from the synthetic
    # base flow: GMRES(100) restarted until it converges or saturates, then BiCGstab(2) from its
    # result (Section 3.1), mixed precision; stop at ||F|| < 1e-9 ||F_0||
    n = 64
    gq = kv.Grid(n, n, n, bc=synth.CC, gr=1e4, pr=0.71, precision=kv.KV_PREC_MIXED)
    S = torch.from_numpy(np.stack(synth.base_flow(n, n, n, synth.CC, 11900))).cuda()
    _, f0 = gq.newton_residual(S)
    V = torch.empty((101, 4) + gq.shape, dtype=torch.float64, device="cuda")
    work = torch.empty((10, 4) + gq.shape, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = gq.newton(S, V, work, max_newton=12, tol=1e-9 * f0, gmres_m=100, gmres_max_restarts=100, lin_tol=1e-10,
                   gmres_sat=0.99, bicg_max_iter=300)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    out["newton64"] = {"workload": "64^3 CC, Gr = 1e4, Pr = 0.71: steady state by Newton's method from the synthetic "
                                   "base flow; GMRES(100) restarted until converged or saturated, then BiCGstab(2) "
                                   "(at most 300 iterations); mixed precision",
                       "value": st.matvecs / t, "unit": "Krylov-vector evals/s inside the solves", "seconds": t,
                       "newton_iterations": st.iterations, "converged": bool(st.converged), "matvecs": st.matvecs,
                       "gmres_restarts": st.gmres_restarts, "bicg_iterations": st.bicg_iterations,
                       "bicg_rejected": st.bicg_rejected,
                       "res_norms": [float(r) for r in st.res_norm[:st.n_res]]}
    del V, work, S, gq
    torch.cuda.empty_cache()
    # the same Krylov vector on the grid stretched by Eq (22) at the steepest a = 0.12 of Section
    # 3.2 (FP64: per-axis weight tables, numerically computed eigenpairs of Eq (15))
    g = kv.Grid(w.nx, w.ny, w.nz, bc=w.bc, gr=w.gr, pr=w.pr, precision=kv.KV_PREC_FP64, stretch=0.12)
    g.set_base_flow(torch.from_numpy(np.stack(base_np)).cuda())
    x = torch.from_numpy(x_np[0]).cuda()
    y = g.empty(4)
    t = timed(lambda: g.krylov_vector(x, y), reps=5)
    out["stretched_fp64"] = {"workload": f"{w.name} on the grid stretched by Eq (22), a = 0.12; FP64",
                             "value": 1.0 / t, "unit": UNIT, "ms_per_vector": t * 1e3}
    y64 = y.clone()
    del g
    torch.cuda.empty_cache()
    # the same in mixed precision (the operator reads the plus coefficients)
    g = kv.Grid(w.nx, w.ny, w.nz, bc=w.bc, gr=w.gr, pr=w.pr, precision=kv.KV_PREC_MIXED, stretch=0.12)
    g.set_base_flow(torch.from_numpy(np.stack(base_np)).cuda())
    t = timed(lambda: g.krylov_vector(x, y), reps=5)
    err = (torch.linalg.vector_norm(y - y64) / torch.linalg.vector_norm(y64)).item()
    out["stretched_mixed"] = {"workload": f"{w.name} on the grid stretched by Eq (22), a = 0.12; mixed precision",
                              "value": 1.0 / t, "unit": UNIT, "ms_per_vector": t * 1e3, "rel_err_vs_fp64": err,
                              "tuning": g.tuning()}
    del g, y64
    torch.cuda.empty_cache()
    # the same Krylov vector with first-order upwind advection (the descriptor's option), FP64
    # and mixed precision (the double-float operator that reads the plus coefficients)
    g = kv.Grid(w.nx, w.ny, w.nz, bc=w.bc, gr=w.gr, pr=w.pr, precision=kv.KV_PREC_FP64,
                advection=kv.KV_ADV_UPWIND)
    g.set_base_flow(torch.from_numpy(np.stack(base_np)).cuda())
    t = timed(lambda: g.krylov_vector(x, y), reps=5)
    out["upwind_fp64"] = {"workload": f"{w.name} with first-order upwind advection; FP64",
                          "value": 1.0 / t, "unit": UNIT, "ms_per_vector": t * 1e3}
    y64 = y.clone()
    del g
    torch.cuda.empty_cache()
    g = kv.Grid(w.nx, w.ny, w.nz, bc=w.bc, gr=w.gr, pr=w.pr, precision=kv.KV_PREC_MIXED,
                advection=kv.KV_ADV_UPWIND)
    g.set_base_flow(torch.from_numpy(np.stack(base_np)).cuda())
    t = timed(lambda: g.krylov_vector(x, y), reps=5)
    err = (torch.linalg.vector_norm(y - y64) / torch.linalg.vector_norm(y64)).item()
    out["upwind_mixed"] = {"workload": f"{w.name} with first-order upwind advection; mixed precision",
                           "value": 1.0 / t, "unit": UNIT, "ms_per_vector": t * 1e3, "rel_err_vs_fp64": err,
                           "tuning": g.tuning()}
    del g, x, y, y64
    torch.cuda.empty_cache()
    return out


def cpu_baselines(w, out):
    """The oracle on the host cores beside the GPU figures: the benchmark workload on all cores
    (best of 3 after a warm-up), a 100^3 workload on one core (best of 3 after a warm-up), and
    one bounded sample each beside the Newton, stretched-grid and upwind lines (when present in out)."""
    if "newton64" in out:  # the oracle beside the Newton line: one bounded GMRES cycle
        try:
            cmd = [sys.executable, "-m", "oracle.bench_cpu", "--newton-cycle", "20"]
            r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
            if r.returncode != 0:
                raise RuntimeError(r.stderr[-500:])
            rc = json.loads(r.stdout.strip().splitlines()[-1])
            out["newton64"]["cpu_baseline"] = {"value": rc["value"], "unit": rc["unit"], "cores": rc["cores"],
                                               "kind": "oracle", "sample": f"{rc['sample']} ({rc['seconds']:.1f} s)"}
        except Exception as e:
            out["newton64"]["cpu_baseline"] = {"value": None, "kind": "oracle", "sample": f"failed: {e}"[:300]}
    if "stretched_fp64" in out:  # the oracle beside the stretched line: one evaluation
        try:
            rc = cpu_baseline(w.name, 1, 0, timeout=120, extra=["--stretch", "0.12"])
            out["stretched_fp64"]["cpu_baseline"] = {
                "value": rc["value"], "unit": UNIT, "cores": rc["cores"], "kind": "oracle",
                "sample": f"1 FP64 oracle Krylov-vector evaluation of {w.name} stretched by Eq (22), a = 0.12 "
                          f"({rc['seconds']:.1f} s on {rc['cores']} host threads; the grid set-up, "
                          f"{rc['setup_seconds']:.1f} s, not timed)"}
        except Exception as e:
            out["stretched_fp64"]["cpu_baseline"] = {"value": None, "kind": "oracle", "sample": f"failed: {e}"[:300]}
    if "upwind_fp64" in out:  # the oracle beside the upwind line: one evaluation
        try:
            rc = cpu_baseline(w.name, 1, 0, timeout=120, extra=["--adv", "1"])
            out["upwind_fp64"]["cpu_baseline"] = {
                "value": rc["value"], "unit": UNIT, "cores": rc["cores"], "kind": "oracle",
                "sample": f"1 FP64 oracle Krylov-vector evaluation of {w.name} with upwind advection "
                          f"({rc['seconds']:.1f} s on {rc['cores']} host threads)"}
        except Exception as e:
            out["upwind_fp64"]["cpu_baseline"] = {"value": None, "kind": "oracle", "sample": f"failed: {e}"[:300]}
    try:
        r = cpu_baseline(w.name, 1, 1, best_of=3)
        r1 = cpu_baseline("cube100_cc", 1, 1, best_of=3, one_core=True)
        host = r["host"]
        out["cpu_baseline"] = {
            "value": r["value"], "unit": UNIT, "cores": r["cores"], "kind": "oracle",
            "sample": f"FP64 oracle Krylov-vector evaluation of {w.name} on {r['cores']} host threads, best of 3 "
                      f"after 1 warm-up ({', '.join(f'{t:.2f}' for t in r['all_seconds'])} s; Arnoldi "
                      f"orthogonalisation not included); host: nproc {host.get('nproc')}, "
                      f"{host.get('Model name', '?')}, {host.get('Architecture', '?')}",
            "one_core": {"value": r1["value"], "unit": UNIT, "cores": 1, "workload": "cube100_cc",
                         "seconds": r1["seconds"], "best_of": r1["best_of"],
                         "per_cell_rate_scaled_to_256": r1["value"] * 100 ** 3 / 256 ** 3}}
    except Exception as e:  # the baseline is reported, never required
        out["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle",
                               "sample": f"failed: {e}"[:300]}


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist = None
        torch.cuda.set_device(local)

    from paper_1905_11601_gb300 import build as kvbuild
    from paper_1905_11601_gb300 import kv, synth

    kvbuild.build()
    w = synth.WORKLOADS[args.workload]
    base_np, x_np = synth.workload_arrays(w)
    base = torch.from_numpy(np.stack(base_np)).cuda()
    x = torch.from_numpy(x_np[0]).cuda()
    m = args.restart
    results = {}
    y_ref = None
    for prec in ("fp64", "mixed"):
        g = kv.Grid(w.nx, w.ny, w.nz, bc=w.bc, gr=w.gr, pr=w.pr,
                    precision=kv.KV_PREC_MIXED if prec == "mixed" else kv.KV_PREC_FP64)
        g.set_base_flow(base)
        y0, st = g.krylov_vector(x, stats=True)
        if prec == "fp64":
            y_ref = y0.clone()
            err = 0.0
        else:
            err = (torch.linalg.vector_norm(y0 - y_ref) / torch.linalg.vector_norm(y_ref)).item()
            assert st.device_error == 0
        V = torch.zeros((m + 1, 4) + g.shape, dtype=torch.float64, device="cuda")
        V[0] = y0 / torch.linalg.vector_norm(y0)
        del y0
        g.guard(reset=True)
        ms, phases, clk, nqs, (steps_seen, second), runs = arnoldi_run(
            g, V, m, args.steps, args.warmup, dist, clocks_index=local if (rank == 0 and prec == "mixed") else None)
        # the device-side SIMPLE test of every Krylov vector of the run (warm-up, timed and
        # phase-timing passes), read after the timed region
        guard = g.guard(reset=True)
        # the Krylov vector alone (no orthogonalisation), same inputs, CUDA events
        yk = torch.empty_like(x)
        kv_ms = timed(lambda: g.krylov_vector(x, yk), reps=max(3, args.steps // 2), warm=2) * 1e3
        del yk
        results[prec] = {"g": g, "ms": ms, "phases": phases, "clocks": clk, "err": err, "nq": nqs,
                         "rel_div": st.rel_div, "value": whole_job_rate(args.steps, world, ms / 1000.0),
                         "guard": guard, "second_updates": [second, steps_seen], "kv_ms": kv_ms, "runs": runs}
        del V
        if prec == "fp64":
            del g
            results[prec].pop("g")
            torch.cuda.empty_cache()

    g = results["mixed"]["g"]
    # End to end through the host-buffer entry points (pinned host memory, every vector's copies
    # inside the timed region): the streamed form (copies overlapping the evaluations) is the
    # e2e value; one kv_krylov_vector_host call per vector is reported beside it.
    # (one untimed pass over every buffer first; the median of three timed passes is the value,
    # all three are reported: the host link's rate varies with what else the host is doing)
    ne = args.e2e_steps
    Xh = torch.from_numpy(np.stack([x_np[0]] * ne).reshape(ne, -1)).pin_memory()
    Yh = torch.empty_like(Xh).pin_memory()
    g.krylov_vector_host_stream(Xh, Yh)
    torch.cuda.synchronize()
    e2e_runs = []
    for _ in range(3):
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        g.krylov_vector_host_stream(Xh, Yh)
        e2e_runs.append(whole_job_rate(ne, world, max_over_ranks(time.perf_counter() - t0, dist)))
    e2e_value = sorted(e2e_runs)[1]
    xh, yh = Xh[0], Yh[0]
    g.krylov_vector_host(xh, yh)
    torch.cuda.synchronize()
    single_runs = []
    for _ in range(3):
        t0 = time.perf_counter()
        for _ in range(ne):
            g.krylov_vector_host(xh, yh)
        single_runs.append(whole_job_rate(ne, world, max_over_ranks(time.perf_counter() - t0, dist)))
    e2e_single = sorted(single_runs)[1]
    vec_bytes = xh.numel() * 8

    mx = results["mixed"]
    fp = results["fp64"]
    roof = roofline(mx["phases"], w, "mixed", args.steps, mx["nq"], mx["g"].tuning())
    launches = int(sum(p["launches"] for p in mx["phases"].values()))
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    out = {"metric": METRIC, "value": mx["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": mx["ms"] / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_MIXED,
           "data": "synthetic (seeded base flow and vectors)", "config": workload_desc(w, m, "mixed"),
           "impl": "ours",
           "step": "one Arnoldi step = one Krylov-vector evaluation + classical Gram-Schmidt applied twice, the "
                   "second projection and the normalisation of each new vector deferred to the next step "
                   "(kv_arnoldi_run over the steps between restarts, one synchronisation per call); value = "
                   "steps/s = Krylov vectors/s including their orthogonalisation",
           "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": vec_bytes,
                   "d2h_bytes_per_step": vec_bytes,
                   "path": f"kv_krylov_vector_host_stream over {ne} vectors, mixed precision (pinned host X and Y; "
                           f"copy-in of the next and copy-out of the previous vector overlap each evaluation)",
                   "single_call_value": e2e_single, "runs": e2e_runs, "single_call_runs": single_runs,
                   "statistic": "median of 3 timed passes after one untimed pass"},
           "gpu_launches": launches, "roofline": roof, "clocks": mx["clocks"], "tuning": mx["g"].tuning()}
    if not args.no_extras:
        out.update(extras(base_np, x_np, w, kv, synth))
    if world == 1 and not args.no_cpu_baseline:
        cpu_baselines(w, out)
    # the figures the headline rests on, last on the line (a truncated record keeps its end)
    out["simple_guard"] = dict(mx["guard"], tol=1e-11,
                               note="device-side SIMPLE test (max|Dv| h_min / max|v|) of every Krylov vector in the "
                                    "mixed run, timed steps included; read after the timed region")
    out["second_gs_update"] = {"steps": mx["second_updates"][1], "with_second_update": mx["second_updates"][0],
                               "note": "the phase-timing pass over the timed basis sizes; the delayed form applies "
                                       "every step's second projection (in the next step's sweeps)"}
    # the operator phase's own roofline (the line's roofline object is the dominant phase's)
    out["roofline_operator"] = roofline({"stencil": mx["phases"]["stencil"]}, w, "mixed", args.steps,
                                        mx["nq"], mx["g"].tuning())
    out["phases"] = {k: {"ms_per_step": v["ms"] / args.steps, "share": v["share"],
                         "launches_per_step": v["launches"] / args.steps} for k, v in mx["phases"].items()}
    # each HBM-bound phase's algorithmic bytes per step over its time, as a fraction of the copy
    # bandwidth (the bytes of the roofline function; the tensor-core phase is not HBM-bound)
    hbm_peak = measured_peaks()[0]
    L = 4 * (w.nx + 2) * (w.ny + 2) * (w.nz + 2)
    n3 = w.nx * w.ny * w.nz
    nqm = sum(mx["nq"]) / len(mx["nq"]) if mx["nq"] else 0.0
    algo = {"stencil": 12 * 8.0 * n3, "divergence": (4 * 8.0 + 6.0) * n3, "correct": 7 * 8.0 * n3,
            "refine": (2 * 8.0 + 6.0) * n3, "gs_dots": 8.0 * L * (nqm + 1), "gs_update": 8.0 * L * (nqm + 3)}
    for k, byts in algo.items():
        ph = out["phases"].get(k)
        if ph and ph["ms_per_step"] > 0:
            ph["hbm_frac"] = byts / (ph["ms_per_step"] / 1e3) / 1e9 / hbm_peak
    # The whole step against its bounds: the sum over phases of the time at the bound, over the
    # measured step time. Algorithmic work: the Krylov vector's streaming steps move 13 fields
    # (read x and the base state, write y and p); the Poisson solves are 12 N^4 flops per solve
    # for each of the 6 BF16 slice products, at the sustained tensor rate; the Gram-Schmidt
    # sweeps stream the basis, the provisional vector and its image as they run (the delayed form:
    # nq + 1 vectors for the inner products and nq + 3 for the update per step, and the last
    # vector's two sweeps, (J + 1) + (J + 2), once per run). The refinement residual and the other
    # intermediates are implementation traffic, with no time at the bound.
    bf16, bf16_src = bf16_peak()
    tpd = out["phases"].get("tpd", {})
    sweeps = tpd.get("launches_per_step", 12.0) / 6.0
    nqs_t = mx["nq"]
    ends = [nq for i, nq in enumerate(nqs_t) if i + 1 == len(nqs_t) or nqs_t[i + 1] <= nq]
    final_per_step = sum((J + 1) + (J + 2) for J in ends) / max(len(nqs_t), 1)
    t_min = {"operator + divergence + correction (HBM, 13 fields x 8 B x N^3)": 13 * 8.0 * n3 / (hbm_peak * 1e9),
             "Poisson contractions (tensor, 6 x 12 N^4 flops x sweeps)":
                 6 * 12.0 * w.nx * w.ny * w.nz * (w.nx + w.ny + w.nz) / 3.0 * sweeps / (bf16 * 1e12),
             "Gram-Schmidt sweeps (HBM, basis and vector streams)":
                 8.0 * L * ((nqm + 1) + (nqm + 3) + final_per_step) / (hbm_peak * 1e9)}
    t_sum = sum(t_min.values())
    kv_min = t_sum - t_min["Gram-Schmidt sweeps (HBM, basis and vector streams)"]
    out["roofline_step"] = {
        "frac": t_sum / (out["ms_per_step"] / 1e3),
        "t_min_ms": {k: v * 1e3 for k, v in t_min.items()}, "t_measured_ms": out["ms_per_step"],
        "krylov_vector_frac": kv_min / (mx["kv_ms"] / 1e3), "krylov_vector_ms": mx["kv_ms"],
        "peaks": {"hbm_gbs": hbm_peak, "bf16_tflops": bf16, "source": bf16_src},
        "what": "sum over phases of (algorithmic work / peak) over the measured time; the Krylov vector's "
                "intermediates (v*, b, phi and the refinement residual) count as implementation traffic"}
    out["fp64_plain"] = {"value": fp["value"], "ms_per_step": fp["ms"] / args.steps,
                         "krylov_vector_ms": fp["kv_ms"],
                         "roofline": roofline(fp["phases"], w, "fp64", args.steps, fp["nq"]),
                         "phases": {k: {"ms_per_step": v["ms"] / args.steps, "share": v["share"]}
                                    for k, v in fp["phases"].items()}}
    out["krylov_vector_only"] = {"value": 1e3 / mx["kv_ms"], "unit": UNIT, "ms": mx["kv_ms"],
                                 "fp64_value": 1e3 / fp["kv_ms"], "fp64_ms": fp["kv_ms"],
                                 "speedup_of_mixed": fp["kv_ms"] / mx["kv_ms"],
                                 "what": "kv_krylov_vector alone on the benchmark workload, inputs in HBM"}
    out["speedup_of_mixed_arnoldi_step"] = mx["value"] / fp["value"]
    out["rel_err_vs_fp64"] = mx["err"]
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def run_single(args):
    """Two Krylov-vector evaluations of the workload (for a profiler's kernel capture): the first
    with statistics, the second without (the bench's own path)."""
    import numpy as np
    import torch

    from paper_1905_11601_gb300 import build as kvbuild
    from paper_1905_11601_gb300 import kv, synth

    kvbuild.build()
    if args.single == "mixed-newton":
        n = 64
        g = kv.Grid(n, n, n, bc=synth.CC, gr=1e4, pr=0.71, precision=kv.KV_PREC_MIXED)
        S = torch.from_numpy(np.stack(synth.base_flow(n, n, n, synth.CC, 11900))).cuda()
        V = torch.empty((31, 4) + g.shape, dtype=torch.float64, device="cuda")
        work = torch.empty((10, 4) + g.shape, dtype=torch.float64, device="cuda")
        st = g.newton(S, V, work, max_newton=2, tol=0.0, gmres_m=30, gmres_max_restarts=1, lin_tol=1e-10,
                      gmres_sat=0.99, bicg_max_iter=2)
        torch.cuda.synchronize()
        print(f"single mixed-newton 64^3: {st.iterations} corrections, {st.matvecs} Krylov vectors")
        return
    w = synth.WORKLOADS[args.workload]
    base_np, x_np = synth.workload_arrays(w)
    g = kv.Grid(w.nx, w.ny, w.nz, bc=w.bc, gr=w.gr, pr=w.pr,
                precision=kv.KV_PREC_FP64 if args.single == "fp64" else kv.KV_PREC_MIXED,
                advection=kv.KV_ADV_UPWIND if args.advection == "upwind" else kv.KV_ADV_CENTRAL)
    if args.operator and args.single != "fp64":
        variant, planes = (int(v) for v in args.operator.split(","))
        g.set_tuning((32, 8), variant, (0 if variant else 32, planes))
    g.set_base_flow(torch.from_numpy(np.stack(base_np)).cuda())
    x = torch.from_numpy(x_np[0]).cuda()
    y, st = g.krylov_vector(x, stats=True)  # statistics for the line printed below
    y = g.krylov_vector(x)                   # the evaluation a profiler captures (no statistics)
    if args.single in ("mixed-arnoldi", "mixed-arnoldi-run"):
        V = torch.zeros((9, 4) + g.shape, dtype=torch.float64, device="cuda")
        V[0] = y / torch.linalg.vector_norm(y)
        if args.single == "mixed-arnoldi-run":
            g.arnoldi_run(V, 0, 8)
        else:
            for j in range(8):
                g.arnoldi_step(V, j)
    torch.cuda.synchronize()
    print(f"single {args.single} {w.name}: rel_div {st.rel_div:.2e} device_error {st.device_error}")


def main():
    args = parse_args()
    if args.single:
        run_single(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
