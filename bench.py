#!/usr/bin/env python
"""MINRES-CG throughput on one GB300: solves/s at true relative residual 1e-10.

Workload: 3D 7-point Dirichlet Laplacian on a 128^3 grid (n = 2,097,152,
nnz = 14,581,760) shifted midway between its 10th and 11th eigenvalues
(k = 10 negative eigenvalues), x* = uniform[-1, 1] (seed 1), b = A x*.
One step = one full solve from x0 = 0: outer FP64 MINRES, inner CG on
M_mr = A + 2 V|Lambda|V^T with inner_tol 1e-3, stopping at FP64 true relative
residual <= 1e-10.  The headline is the mixed-precision solver (FP32 inner CG,
FP64 outer); the plain FP64 solver is measured in the same run.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs an independent replica (no data-path
collective); value = solves of all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "solves/s & SpMV HBM GB/s at true rel. residual 1e-10, mixed vs FP64, 1xGB300"
WORKLOAD = "lap3d_128^3_k10: 3D 7-pt Laplacian 128^3 (n=2,097,152) shifted to 10 negative eigenvalues, 1 RHS"
BATCH_WORKLOAD = ("batch64: 64 x 2D 5-pt Laplacian, sides U{100..400}, k_i U{1..16} (cluster-rounded), "
                  "RHS uniform[-1,1], seed 3, one batched solve per step")
SHIFTED_WORKLOAD = ("shifted64: 3D 7-pt Laplacian 160^3 (n=4,096,000), 16 shifts with k_j U{1..30} "
                    "cluster-rounded (seed 4), 4 RHS each, one 64-column block")
OUTER_TOL, INNER_TOL = 1e-10, 1e-3
CPU_SAMPLE_ITERS = 120  # inner iterations of the oracle's solve timed for the CPU baseline


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["lap3d_128", "lap2d_64", "lap3d_128_near", "saddle", "batch64",
                                           "shifted64"],
                    default="lap3d_128",
                    help="lap3d_128: the headline single-system workload; lap3d_128_near: the same matrix with "
                         "sigma close to lambda_10 (for --mcg smw, MINRES-CG*); batch64: 64 independent uneven "
                         "2D systems (sides 100..400, k_i 1..16, seed 3) solved as one batch; shifted64: 16 "
                         "shifts x 4 RHS of the 160^3 Laplacian as one right-hand-side block")
    ap.add_argument("--inner-tol", type=float, default=INNER_TOL,
                    help="relative recursive-residual tolerance of every inner CG solve (default 1e-3); the CPU "
                         "baseline of a sampled workload is scaled only by a count recorded at the same tolerance")
    ap.add_argument("--mcg", choices=["identity", "jacobi", "smw"], default="identity",
                    help="inner preconditioner of the single-system workloads: identity (default), Jacobi on "
                         "M_mr, or smw, the MINRES-CG* form diag(A)^-1 - 2 V Lambda^-1 V^T (Sec. 2.1)")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers

def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    return ws, rank, local


def replica_throughput(ms_local, ok_local, ws, dev):
    """Whole-job throughput of independent replicas: the solves that met the
    tolerance on all ranks over the slowest rank's time.  Returns (max ms,
    total ok, solves/s)."""
    ms = max_over_ranks(ms_local, ws, dev)
    ok = sum_over_ranks(ok_local, ws, dev)
    return ms, ok, ok / (ms / 1000.0)


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws, dev):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, ws, dev):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0])); mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


KERNEL_SOURCES = ["paper_1805_12417_gb300/csrc/cg_impl.cuh", "paper_1805_12417_gb300/csrc/common.cuh"]
TRAFFIC_RECORDS = "profiles/traffic.json"


def step_a_kernel_name(cfg, prec="float"):
    """Name of the step-a kernel a launch configuration runs, as ncu prints it."""
    var, kb = cfg["step_a_variant"], cfg["k_bucket"]
    if var in (9, 10, 12, 13):
        mb, pipe = {9: (2, 0), 10: (3, 0), 12: (2, 1), 13: (3, 1)}[var]
        return f"cg_step_a_pg_staged_kernel<{prec}, {kb}, {mb}, {pipe}>"
    if var == 11:
        return f"cg_step_a_pg_kernel<{prec}, {kb}>"
    if var == 8:
        return f"cg_step_a_staged_kernel<{prec}, {kb}, 3, 0, 1>"
    if var >= 5:
        mb, pipe = {5: (2, 0), 6: (4, 0), 7: (2, 1)}[var]
        return f"cg_step_a_staged_kernel<{prec}, {kb}, {mb}, {pipe}, 0>"
    return f"cg_step_a_kernel<{prec}, {kb}, {var}>"


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu record
    (profiles/traffic.json), if it was taken on the current kernel sources
    (else None)."""
    path = os.path.join(ROOT, TRAFFIC_RECORDS)
    try:
        with open(path) as f:
            recs = json.load(f)["records"]
    except (OSError, ValueError, KeyError):
        return None
    want = kernel_source_hash()
    for r in recs:
        if r.get("kernel") == kernel and r.get("source_sha256") == want:
            return int(r["bytes_per_launch"])
    return None


def measured_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def full_solve_inner_iters(name, mcg="identity"):
    """Inner iterations of a whole FP64 oracle solve, as recorded by
    oracle/record_counts.py (None when that workload was not recorded)."""
    path = os.path.join(ROOT, "oracle", "full_solve_counts.json")
    k = f"{name}|outer={OUTER_TOL:g}|inner={INNER_TOL:g}" + ("" if mcg == "identity" else f"|mcg={mcg}")
    try:
        with open(path) as f:
            rec = json.load(f)
        return int(rec[k]["inner_iters_total"])
    except Exception:
        return None


def single_system(name):
    """(problem, description) of a single-system workload."""
    from gen import lap2d_64_k4, lap3d_128_k10, lap3d_128_k10_near, saddle_96_b20x64
    if name == "saddle":
        return saddle_96_b20x64(), (
            "saddle_96^3_B20x64: [K B^T; B 0], K 27-pt log-normal(0,1) SPD stencil on 96^3, B 20 rows x 64 "
            "uniform[-1,1] entries (n=884,756, 20 negative eigenvalues), seed 2, 1 RHS")
    if name == "lap2d_64":
        return lap2d_64_k4(), (
            "lap2d_64x64_k4: 2D 5-pt Laplacian 64^2 (n=4,096) shifted to 4 negative eigenvalues, 1 RHS; "
            "L2-resident and latency-bound: read solves/s and launches per solve, not the HBM fraction")
    if name == "lap3d_128_near":
        return lap3d_128_k10_near(), (
            "lap3d_128^3_k10_near: the lap3d_128 matrix with sigma at lambda_10 + 0.05 (lambda_11 - "
            "lambda_10), so the 10 negative eigenvalues are the smallest in modulus, 1 RHS")
    return lap3d_128_k10(), WORKLOAD


def cpu_baseline(p, mcg="identity"):
    """The oracle as it stands (serial C, FP64) with the same inner
    preconditioner: a whole solve for small workloads (up to 100,000 rows),
    else its first CPU_SAMPLE_ITERS inner iterations scaled to one full solve
    by the oracle's own recorded count (value None when none is recorded)."""
    import oracle as O
    code = {"identity": O.MCG_IDENTITY, "jacobi": O.MCG_JACOBI, "smw": O.MCG_SMW}[mcg]
    s = O.System.from_problem(p)
    if p.n <= 100_000:
        t = time.perf_counter()
        r = O.minres_cg(s, p.b, outer_tol=OUTER_TOL, inner_tol=INNER_TOL, mcg=code)
        dt = time.perf_counter() - t
        return {"value": 1.0 / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
                "sample": f"one full FP64 oracle solve ({r.inner_iters_total} inner iterations, {dt:.2f} s)",
                "seconds": round(dt, 3)}
    t = time.perf_counter()
    r = O.minres_cg(s, p.b, outer_tol=OUTER_TOL, inner_tol=INNER_TOL, max_iters=CPU_SAMPLE_ITERS, mcg=code)
    dt = time.perf_counter() - t
    n_full = full_solve_inner_iters(p.name, mcg)
    head = f"first {r.inner_iters_total} inner CG iterations of the FP64 oracle solve ({dt:.1f} s)"
    if n_full is None:
        return {"value": None, "unit": "solves/s", "cores": 1, "kind": "oracle", "seconds": round(dt, 2),
                "sample": head + "; no whole oracle solve of this workload is recorded to scale them by"}
    return {"value": r.inner_iters_total / n_full / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": head + f", scaled by the {n_full} inner iterations of a whole oracle solve",
            "seconds": round(dt, 2)}


def cpu_baseline_batch(ps, budget_s=20.0):
    """The oracle on an uneven batch: whole solves of the systems in batch
    order until budget_s has passed (at least one); solves/s of that sample."""
    import oracle as O
    t0 = time.perf_counter()
    done, iters = 0, 0
    for p in ps:
        r = O.minres_cg(O.System.from_problem(p), p.b, outer_tol=OUTER_TOL, inner_tol=INNER_TOL)
        done += 1
        iters += r.inner_iters_total
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "solves/s", "cores": 1, "kind": "oracle", "seconds": round(dt, 2),
            "sample": f"whole FP64 oracle solves of the first {done} of {len(ps)} systems in batch order "
                      f"({sum(p.n for p in ps[:done])} rows, {iters} inner iterations, {dt:.1f} s)"}


def cpu_baseline_shifted(fam):
    """The oracle on a shifted family, sampled on column 0 (shift 0, right-hand
    side 0) as a stand-alone system: its first CPU_SAMPLE_ITERS inner
    iterations, scaled by the inner-iteration count of a whole oracle solve of
    that column (value None when none is recorded).  Columns differ in k_j
    and sigma_j, so this is a per-column rate of one representative column."""
    import oracle as O
    p = fam.column_problem(0)
    t = time.perf_counter()
    r = O.minres_cg(O.System.from_problem(p), p.b, outer_tol=OUTER_TOL, inner_tol=INNER_TOL,
                    max_iters=CPU_SAMPLE_ITERS)
    dt = time.perf_counter() - t
    n_full = full_solve_inner_iters(p.name)
    head = (f"first {r.inner_iters_total} inner CG iterations of the FP64 oracle solve of column 0 "
            f"(shift 0, k = {p.k}; {dt:.1f} s)")
    if n_full is None:
        return {"value": None, "unit": "solves/s", "cores": 1, "kind": "oracle", "seconds": round(dt, 2),
                "sample": head + "; no whole oracle solve of that column is recorded to scale them by"}
    return {"value": r.inner_iters_total / n_full / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "seconds": round(dt, 2),
            "sample": head + f", scaled by the {n_full} inner iterations of a whole oracle solve of that column: "
                             f"column solves per second"}


# ------------------------------------------------------------------ reference arm (the oracle)

def run_reference(args, ws, rank):
    """The oracle, as it stands, on this arm's workload: each step is one
    bounded sample (cpu_baseline*)."""
    if rank != 0:
        return
    if args.workload == "batch64":
        from gen import batch64_lap2d
        ps = batch64_lap2d()
        sample, desc = (lambda: cpu_baseline_batch(ps)), BATCH_WORKLOAD
    elif args.workload == "shifted64":
        from gen import shifted_lap3d_160
        fam = shifted_lap3d_160()
        sample, desc = (lambda: cpu_baseline_shifted(fam)), SHIFTED_WORKLOAD
    else:
        p, desc = single_system(args.workload)
        sample = lambda: cpu_baseline(p, args.mcg)  # noqa: E731
    vals = []
    for i in range(args.warmup + args.steps):
        cb = sample()
        if i >= args.warmup:
            vals.append(cb["value"])
    v = None if any(x is None for x in vals) else statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": (1000.0 / v) if v else None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "inner_prec": args.mcg, "outer_tol": OUTER_TOL, "inner_tol": INNER_TOL,
                       "parallelism": "rank 0 only (CPU oracle)"},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def run_batch64(args, ws, rank, local):
    """64 independent uneven 2D shifted Laplacians solved as one batch; a step is
    one batched solve of all 64 systems."""
    import torch

    from gen import batch64_lap2d
    from paper_1805_12417_gb300 import build as _b
    _b.build()
    import paper_1805_12417_gb300 as m

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    ps = batch64_lap2d()
    B = np.concatenate([p.b for p in ps])
    Bd = torch.from_numpy(B).to(dev)
    Xd = torch.zeros_like(Bd)
    out = {}
    for name, prec in (("mixed", m.MIXED_FP32), ("fp64", m.FP64)):
        with m.Batch(ps, precision=prec, validate=False, stream=stream.cuda_stream) as bt:
            for _ in range(args.warmup):
                Xd.zero_()
                bt.solve(Bd, Xd, outer_tol=OUTER_TOL, inner_tol=INNER_TOL)
            barrier(ws)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ck = Clocks(local) if (rank == 0 and name == "mixed") else None
            if ck:
                ck.__enter__()
            e0.record(stream)
            ok, infos = 0, None
            for _ in range(args.steps):
                Xd.zero_()
                _, st, infos = bt.solve(Bd, Xd, outer_tol=OUTER_TOL, inner_tol=INNER_TOL)
                ok += sum(1 for i in infos if i.status == m.OK and i.true_relres <= OUTER_TOL)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            barrier(ws)
            if ck:
                ck.__exit__(None, None, None)
            ms = max_over_ranks(e0.elapsed_time(e1), ws, dev)
            ok = sum_over_ranks(ok, ws, dev)
            w = 4 if prec == m.MIXED_FP32 else 8
            # algorithmic bytes of the inner iterations actually run (both CG kernels)
            byts = sum(i.inner_iters_total * (p.nnz * (w + 4) + 10 * p.n * w + 2 * p.k * p.n * w)
                       for i, p in zip(infos, ps))
            out[name] = {"value": ok / (ms / 1000.0), "ms_per_step": ms / args.steps,
                         "inner_gbs": byts / (ms / args.steps * 1e-3) / 1e9, "launches": infos[0].kernel_launches,
                         "inner_iters_max": max(i.inner_iters_total for i in infos),
                         "outer_iters_max": max(i.outer_iters for i in infos),
                         "clocks": ck.summary() if ck else None}
            if name == "mixed":
                b_h = torch.from_numpy(B.copy()).pin_memory()
                x_h = torch.zeros(len(B), dtype=torch.float64).pin_memory()
                t0 = time.perf_counter()
                ok_e2e = 0
                for _ in range(args.steps):
                    x_h.zero_()
                    _, st, inf = bt.solve(b_h, x_h, outer_tol=OUTER_TOL, inner_tol=INNER_TOL)
                    ok_e2e += sum(1 for i in inf if i.status == m.OK and i.true_relres <= OUTER_TOL)
                out["e2e"] = {"value": ok_e2e / (time.perf_counter() - t0), "unit": "solves/s",
                              "h2d_bytes_per_step": 2 * len(B) * 8, "d2h_bytes_per_step": len(B) * 8}
    if rank == 0:
        peak, kind = measured_peak_gbs()
        mx = out["mixed"]
        line = {"metric": METRIC, "value": mx["value"], "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": mx["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32 inner CG + f64 outer MINRES",
                "data": "synthetic",
                "config": {"workload": BATCH_WORKLOAD,
                           "systems": len(ps), "rows": int(len(B)), "outer_tol": OUTER_TOL, "inner_tol": INNER_TOL,
                           "l2": "inputs larger than L2", "parallelism": "replicas" if ws > 1 else "single GPU"},
                "roofline": {"kernel": "whole inner loop (batched step a + step b)", "bound": "hbm",
                             "achieved": round(mx["inner_gbs"], 1), "peak": peak, "unit": "GB/s",
                             "frac": round(mx["inner_gbs"] / peak, 4), "traffic": None,
                             "peak_kind": f"{kind} copy bandwidth"},
                "fp64": out["fp64"], "mixed": mx, "mixed_vs_fp64_speedup": mx["value"] / out["fp64"]["value"],
                "e2e": out["e2e"], "gpu_launches": int(mx["launches"] * args.steps), "clocks": mx["clocks"],
                "cpu_baseline": cpu_baseline_batch(ps) if (ws == 1 and not args.no_cpu_baseline) else None}
        print(json.dumps(line), flush=True)


def run_shifted64(args, ws, rank, local):
    """16 shifts x 4 right-hand sides of the 160^3 Laplacian solved as one
    right-hand-side block; a step is one solve of all 64 columns."""
    import torch

    from gen import shifted_lap3d_160
    from paper_1805_12417_gb300 import build as _b
    _b.build()
    import paper_1805_12417_gb300 as m

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    fam = shifted_lap3d_160()
    Bd = torch.from_numpy(fam.B).to(dev)
    Xd = torch.zeros_like(Bd)
    out = {}
    n, nc = fam.n, fam.ncols
    for name, prec, steps, warm in (("mixed", m.MIXED_FP32, args.steps, args.warmup), ("fp64", m.FP64, 1, 1)):
        with m.Shifted(fam, precision=prec, stream=stream.cuda_stream) as sh:
            for _ in range(warm):
                Xd.zero_()
                sh.solve(Bd, Xd, outer_tol=OUTER_TOL, inner_tol=INNER_TOL)
            barrier(ws)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ck = Clocks(local) if (rank == 0 and name == "mixed") else None
            if ck:
                ck.__enter__()
            e0.record(stream)
            ok, infos = 0, None
            for _ in range(steps):
                Xd.zero_()
                _, st, infos = sh.solve(Bd, Xd, outer_tol=OUTER_TOL, inner_tol=INNER_TOL)
                ok += sum(1 for i in infos if i.status == m.OK and i.true_relres <= OUTER_TOL)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            barrier(ws)
            if ck:
                ck.__exit__(None, None, None)
            ms = max_over_ranks(e0.elapsed_time(e1), ws, dev)
            ok = sum_over_ranks(ok, ws, dev)
            w = 4 if prec == m.MIXED_FP32 else 8
            iters = max(i.inner_iters_total for i in infos)  # lock-step block iterations
            byts = iters * (fam.nnz * (w + 4) + 10 * n * 64 * w + 2 * n * 32 * w)
            xh = Xd.cpu().numpy()
            err = max(float(np.linalg.norm(xh[:, c] - fam.xstar[:, c]) / np.linalg.norm(fam.xstar[:, c]))
                      for c in range(nc))
            out[name] = {"value": ok / (ms / 1000.0), "ms_per_step": ms / steps, "steps": steps,
                         "inner_gbs": byts / (ms / steps * 1e-3) / 1e9, "launches": infos[0].kernel_launches,
                         "inner_iters_max": iters, "outer_iters_max": max(i.outer_iters for i in infos),
                         "max_rel_err_vs_xstar": err, "clocks": ck.summary() if ck else None}
            if name == "mixed":
                b_h = torch.from_numpy(fam.B.copy()).pin_memory()
                x_h = torch.zeros(fam.B.shape, dtype=torch.float64).pin_memory()
                t0 = time.perf_counter()
                ok_e2e = 0
                for _ in range(steps):
                    x_h.zero_()
                    _, st, inf = sh.solve(b_h, x_h, outer_tol=OUTER_TOL, inner_tol=INNER_TOL)
                    ok_e2e += sum(1 for i in inf if i.status == m.OK and i.true_relres <= OUTER_TOL)
                out["e2e"] = {"value": ok_e2e / (time.perf_counter() - t0), "unit": "solves/s",
                              "h2d_bytes_per_step": 2 * n * nc * 8, "d2h_bytes_per_step": n * nc * 8}
    if rank == 0:
        peak, kind = measured_peak_gbs()
        mx = out["mixed"]
        line = {"metric": METRIC, "value": mx["value"], "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": mx["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32 inner CG + f64 outer MINRES",
                "data": "synthetic",
                "config": {"workload": SHIFTED_WORKLOAD,
                           "columns": nc, "outer_tol": OUTER_TOL, "inner_tol": INNER_TOL,
                           "l2": "inputs larger than L2", "parallelism": "replicas" if ws > 1 else "single GPU"},
                "roofline": {"kernel": "whole inner loop (block step a + step b)", "bound": "hbm",
                             "achieved": round(mx["inner_gbs"], 1), "peak": peak, "unit": "GB/s",
                             "frac": round(mx["inner_gbs"] / peak, 4), "traffic": None,
                             "peak_kind": f"{kind} copy bandwidth"},
                "fp64": out["fp64"], "mixed": mx, "mixed_vs_fp64_speedup": mx["value"] / out["fp64"]["value"],
                "e2e": out["e2e"], "gpu_launches": int(mx["launches"] * args.steps), "clocks": mx["clocks"],
                "cpu_baseline": cpu_baseline_shifted(fam) if (ws == 1 and not args.no_cpu_baseline) else None}
        print(json.dumps(line), flush=True)


def main():
    global INNER_TOL
    args = parse()
    INNER_TOL = args.inner_tol
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.workload == "batch64":
        run_batch64(args, ws, rank, local)
        return
    if args.workload == "shifted64":
        run_shifted64(args, ws, rank, local)
        return
    import torch

    from paper_1805_12417_gb300 import build as _b
    _b.build()
    import paper_1805_12417_gb300 as m

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    p, workload = single_system(args.workload)
    b_dev = torch.from_numpy(p.b).to(dev)
    x_dev = torch.zeros(p.n, dtype=torch.float64, device=dev)
    mcg = {"identity": m.MCG_IDENTITY, "jacobi": m.MCG_JACOBI, "smw": m.MCG_SMW}[args.mcg]
    solvers = {prec: m.Solver.from_problem(p, precision=prec, inner_prec=mcg, stream=stream.cuda_stream,
                                           validate=False)
               for prec in (m.MIXED_FP32, m.FP64)}

    def run(prec, steps, warmup, clocks=False):
        s = solvers[prec]
        for _ in range(warmup):
            x_dev.zero_()
            s.solve(b_dev, x_dev, outer_tol=OUTER_TOL, inner_tol=INNER_TOL)
        barrier(ws)
        torch.cuda.synchronize(dev)
        infos = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ck = Clocks(local) if clocks else None
        if ck:
            ck.__enter__()
        e0.record(stream)
        for _ in range(steps):
            x_dev.zero_()
            _, info = s.solve(b_dev, x_dev, outer_tol=OUTER_TOL, inner_tol=INNER_TOL)
            infos.append(info)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(ws)
        if ck:
            ck.__exit__(None, None, None)
        ok = sum(1 for i in infos if i.status == m.OK and i.true_relres <= OUTER_TOL)
        ms, ok, v = replica_throughput(e0.elapsed_time(e1), ok, ws, dev)
        return ms, ok, v, infos, (ck.summary() if ck else None)

    # mixed precision (headline) and plain FP64
    ms_mx, ok_mx, value, inf_mx, clocks = run(m.MIXED_FP32, args.steps, args.warmup, clocks=(rank == 0))
    ms_64, ok_64, fp64_value, inf_64, _ = run(m.FP64, args.steps, max(1, args.warmup))

    # errors against x* (FP64 check on the host)
    x_last = x_dev.cpu().numpy()
    err64 = float(np.linalg.norm(x_last - p.xstar) / np.linalg.norm(p.xstar))
    x_dev.zero_()
    solvers[m.MIXED_FP32].solve(b_dev, x_dev, outer_tol=OUTER_TOL, inner_tol=INNER_TOL)
    xm = x_dev.cpu().numpy()
    errmx = float(np.linalg.norm(xm - p.xstar) / np.linalg.norm(p.xstar))
    rr_mx = float(np.linalg.norm(p.b - p.scipy() @ xm) / np.linalg.norm(p.b))

    # end to end through the C ABI with pinned host buffers (copies inside the call)
    b_h = torch.from_numpy(p.b.copy()).pin_memory()
    x_h = torch.zeros(p.n, dtype=torch.float64).pin_memory()
    sm = solvers[m.MIXED_FP32]
    x_h.zero_()
    sm.solve(b_h, x_h, outer_tol=OUTER_TOL, inner_tol=INNER_TOL)
    barrier(ws)
    t0 = time.perf_counter()
    ok_e2e = 0
    for _ in range(args.steps):
        x_h.zero_()
        _, info = sm.solve(b_h, x_h, outer_tol=OUTER_TOL, inner_tol=INNER_TOL)
        ok_e2e += int(info.status == m.OK and info.true_relres <= OUTER_TOL)
    t_e2e = time.perf_counter() - t0
    t_e2e = max_over_ranks(t_e2e, ws, dev)
    ok_e2e = sum_over_ranks(ok_e2e, ws, dev)

    # dominant kernel: inner-CG step a (SpMV + low-rank term + direction update + dot)
    ta_mx, tb_mx = m.time_inner_kernels(solvers[m.MIXED_FP32].h, 50)
    ta_64, tb_64 = m.time_inner_kernels(solvers[m.FP64].h, 50)
    n, nnz, k = p.n, p.nnz, p.k

    ib = m.launch_config(solvers[m.MIXED_FP32].h)["index_bytes"]

    fused_of = {4: m.launch_config(solvers[m.MIXED_FP32].h)["step_a_variant"] == 8,
                8: m.launch_config(solvers[m.FP64].h)["step_a_variant"] == 8}

    def bytes_a(w):  # A values + column indices, s and p_old read, V read, q and p_new written
        if fused_of[w]:  # one-kernel iteration: r, q, p, z read and r, z, p, q written for the own rows
            return nnz * (w + ib) + k * n * w + 8 * n * w
        return nnz * (w + ib) + 2 * n * w + k * n * w + 2 * n * w + (n * w if args.mcg == "jacobi" else 0)

    def bytes_b(w):  # p, q, z, r read; z, r written (V^T s by recurrence: no V pass)
        if fused_of[w]:
            return 0
        if args.mcg == "jacobi":  # + M_cg^{-1} read, s written
            return 8 * n * w
        if args.mcg == "smw":  # + diag(A)^{-1} and V read, s written
            return 8 * n * w + k * n * w
        return 6 * n * w

    peak, peak_kind = measured_peak_gbs()
    ach_a = bytes_a(4) / (ta_mx * 1e-3) / 1e9
    kname = step_a_kernel_name(m.launch_config(solvers[m.MIXED_FP32].h))
    roof = {"kernel": kname, "bound": "hbm", "achieved": round(ach_a, 1), "peak": peak,
            "unit": "GB/s", "frac": round(ach_a / peak, 4), "traffic": recorded_traffic(kname),
            "peak_kind": f"{peak_kind} copy bandwidth (burst: kernel timed alone)",
            "bytes_per_launch": bytes_a(4), "avg_ms": round(ta_mx, 5)}

    kernels = {
        "mixed": {"step_a_ms": ta_mx, "step_b_ms": tb_mx, "step_a_gbs": bytes_a(4) / (ta_mx * 1e-3) / 1e9,
                  "step_b_gbs": bytes_b(4) / (max(tb_mx, 1e-6) * 1e-3) / 1e9},
        "fp64": {"step_a_ms": ta_64, "step_b_ms": tb_64, "step_a_gbs": bytes_a(8) / (ta_64 * 1e-3) / 1e9,
                 "step_b_gbs": bytes_b(8) / (max(tb_64, 1e-6) * 1e-3) / 1e9},
    }
    launches = sum(i.kernel_launches for i in inf_mx)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(p, args.mcg)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_mx / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 inner CG + f64 outer MINRES", "data": "synthetic",
            "config": {"workload": workload, "n": n, "nnz": nnz, "k": k, "outer_tol": OUTER_TOL,
                       "inner_tol": INNER_TOL, "inner_prec": args.mcg, "precision": "mixed: FP32 inner CG, FP64 outer MINRES",
                       "l2": f"inputs larger than L2 (FP32 A {nnz * 8 / 1e6:.0f} MB + V {k * n * 4 / 1e6:.0f} MB "
                             "+ vectors per inner iteration)",
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "roofline": roof,
            "launch_config": {"mixed": m.launch_config(solvers[m.MIXED_FP32].h),
                              "fp64": m.launch_config(solvers[m.FP64].h)},
            "spmv_hbm_gbs": {"mixed_step_a": round(kernels["mixed"]["step_a_gbs"], 1),
                             "fp64_step_a": round(kernels["fp64"]["step_a_gbs"], 1), "peak": peak},
            "kernels": {kk: {a: round(b, 5) for a, b in v.items()} for kk, v in kernels.items()},
            "fp64": {"value": fp64_value, "unit": "solves/s", "ms_per_step": ms_64 / args.steps,
                     "outer_iters": inf_64[-1].outer_iters, "inner_iters_total": inf_64[-1].inner_iters_total,
                     "true_relres": inf_64[-1].true_relres, "rel_err_vs_xstar": err64},
            "mixed": {"outer_iters": inf_mx[-1].outer_iters, "inner_iters_total": inf_mx[-1].inner_iters_total,
                      "restarts": inf_mx[-1].restarts, "true_relres": inf_mx[-1].true_relres,
                      "true_relres_host_fp64": rr_mx, "rel_err_vs_xstar": errmx},
            "mixed_vs_fp64_speedup": value / fp64_value if fp64_value > 0 else None,
            "e2e": {"value": ok_e2e / t_e2e, "unit": "solves/s", "h2d_bytes_per_step": 2 * n * 8,
                    "d2h_bytes_per_step": n * 8},
            "gpu_launches": int(launches),
            "launches_per_solve": round(launches / max(1, len(inf_mx)), 1),
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    for s in solvers.values():
        s.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
