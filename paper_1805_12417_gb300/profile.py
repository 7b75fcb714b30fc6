"""Small profiling driver: launch the inner-CG iteration kernels on a workload.

Creates a solver for a generated workload and runs `--iters` standalone
launches of each inner-CG kernel (step a, step b) through
mrcg_time_inner_kernels, printing their CUDA-event times.  Few other kernels
run before them (setup only), which keeps an ncu capture of them small:

  python -m paper_1805_12417_gb300.profile --workload lap3d_128 --precision mixed --iters 3

The batch64 and shifted64 workloads instead run one solve of the batch or
shifted-family engine with an inner budget of 100 * --iters iterations and
the inner loop driven from the host (MRCG_INNER_LOOP=host), so that a
profiler sees those engines' kernels.

A profiler slows every launch, which misleads the launch-shape autotuner that
runs at solver creation; `--var-a / --bpsm-a / --bpsm-b` (or MRCG_SHAPE_F32 /
MRCG_SHAPE_F64) fix the shape instead
(the values a normal run reports through mrcg_launch_config).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def workload(name):
    from gen import lap2d_64_k4, lap3d_128_k10, small_3d
    return {"lap3d_128": lap3d_128_k10, "lap2d_64": lap2d_64_k4, "lap3d_small": small_3d}[name]()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="lap3d_128", choices=["lap3d_128", "lap2d_64", "lap3d_small", "batch64", "shifted64"],
                    help="batch64: one batched solve of the 64 uneven 2D systems; shifted64: one solve of a "
                         "64^3 Laplacian family (16 shifts, k_j up to 30, 4 right-hand sides each); both with the "
                         "inner loop driven from the host (MRCG_INNER_LOOP=host), so a profiler sees their kernels")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--var-a", type=int, default=None, help="step-a kernel variant (0-15)")
    ap.add_argument("--bpsm-a", type=int, default=None, help="step-a blocks per SM")
    ap.add_argument("--bpsm-b", type=int, default=None, help="step-b blocks per SM")
    ap.add_argument("--mcg", default="identity", choices=["identity", "jacobi", "smw", "ilu0", "smw_ilu0"],
                    help="inner preconditioner M_cg of the single-system workloads")
    ap.add_argument("--ilu-block", type=int, default=0, help="ILU(0) block rows (0: the library default)")
    a = ap.parse_args(argv)
    # read by the library when the solver is created
    for key, val in (("MRCG_VAR_A", a.var_a), ("MRCG_BPSM_A", a.bpsm_a), ("MRCG_BPSM_B", a.bpsm_b)):
        if val is not None:
            os.environ[key] = str(val)
    import paper_1805_12417_gb300 as m
    prec = m.MIXED_FP32 if a.precision == "mixed" else m.FP64
    if a.workload == "batch64":
        import numpy as np
        from gen import batch64_lap2d
        os.environ["MRCG_INNER_LOOP"] = "host"
        ps = batch64_lap2d()
        B = np.concatenate([q.b for q in ps])
        with m.Batch(ps, precision=prec, validate=False) as bt:
            X, st, infos = bt.solve(B.copy(), outer_tol=1e-10, max_iters=a.iters * 100)
        print(json.dumps({"workload": "batch64", "precision": a.precision, "status": int(st),
                          "inner_iters": int(sum(i.inner_iters_total for i in infos))}))
        return
    if a.workload == "shifted64":
        from gen import shifted_family
        os.environ["MRCG_INNER_LOOP"] = "host"
        fam = shifted_family((64, 64, 64), 16, 4, 30, seed=4, name="lap3d_64^3_16shifts_x4")
        with m.Shifted(fam, precision=prec) as sh:
            X, st, infos = sh.solve(fam.B.copy(), outer_tol=1e-10, max_iters=a.iters * 100)
        print(json.dumps({"workload": "shifted64", "precision": a.precision, "status": int(st),
                          "inner_iters": int(sum(i.inner_iters_total for i in infos))}))
        return
    p = workload(a.workload)
    mcg = {"identity": m.MCG_IDENTITY, "jacobi": m.MCG_JACOBI, "smw": m.MCG_SMW, "ilu0": m.MCG_ILU0,
           "smw_ilu0": m.MCG_SMW_ILU0}[a.mcg]
    with m.Solver.from_problem(p, precision=prec, validate=False, inner_prec=mcg, ilu_block=a.ilu_block) as s:
        ta, tb = m.time_inner_kernels(s.h, a.iters)
        cfg = m.launch_config(s.h)
    print(json.dumps({"workload": p.name, "precision": a.precision, "mcg": a.mcg, "iters": a.iters, "step_a_ms": ta,
                      "step_b_ms": tb, "launch_config": cfg}))


if __name__ == "__main__":
    main()
