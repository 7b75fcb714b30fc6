"""Record the oracle's full-solve iteration counts for the benchmark workloads.

The benchmark's CPU-baseline leg times a bounded sample (the first S inner
iterations) of the oracle's solve and scales it to one full solve with the
inner-iteration total stored here.  It calls only the oracle and the input
generators.  Each record is one whole FP64 oracle solve (minutes each at
2-million-row sizes); records are merged into the JSON file under a lock, so
several invocations may run at once:

    python oracle/record_counts.py                       # every record
    python oracle/record_counts.py lap3d_128_near:smw    # selected records

Record names are `<workload>:<inner preconditioner>`; the key in the file is
`<problem name>|outer=<tol>|inner=<tol>` plus `|mcg=<name>` for an inner
preconditioner other than the identity.
"""
import fcntl
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import gen  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "full_solve_counts.json")
OUTER_TOL, INNER_TOL = 1e-10, 1e-3
MCG = {"identity": O.MCG_IDENTITY, "jacobi": O.MCG_JACOBI, "smw": O.MCG_SMW}
WORKLOADS = {
    "lap2d_64": lambda: gen.lap2d_64_k4(),
    "lap3d_128": lambda: gen.lap3d_128_k10(),
    "lap3d_128_near": lambda: gen.lap3d_128_k10_near(),
    # the saddle's eigenpairs come from a Krylov eigensolver in torch, on the
    # GPU when there is one, else on the CPU (slow; residuals as on the GPU)
    "saddle": lambda: gen.saddle_96_b20x64(),
    # one column of the 160^3 shifted family (shift 0, right-hand side 0) as a
    # stand-alone system: a whole oracle solve of all 64 columns takes a day
    "shifted64_col0": lambda: gen.shifted_lap3d_160().column_problem(0),
}
RECORDS = ["lap2d_64:identity", "lap3d_128:identity", "lap3d_128:jacobi", "lap3d_128:smw",
           "lap3d_128_near:identity", "lap3d_128_near:smw", "saddle:identity", "shifted64_col0:identity"]


def key(name, mcg):
    k = f"{name}|outer={OUTER_TOL:g}|inner={INNER_TOL:g}"
    return k if mcg == "identity" else f"{k}|mcg={mcg}"


def merge(k, v):
    with open(OUT + ".lock", "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        rec = {}
        if os.path.exists(OUT):
            with open(OUT) as f:
                rec = json.load(f)
        rec[k] = v
        with open(OUT, "w") as f:
            json.dump(rec, f, indent=1, sort_keys=True)
            f.write("\n")


def main(names):
    problems = {}
    for r in names:
        wl, mcg = r.split(":")
        if wl not in problems:
            problems[wl] = WORKLOADS[wl]()
        p = problems[wl]
        s = O.System.from_problem(p)
        t = time.perf_counter()
        res = O.minres_cg(s, p.b, outer_tol=OUTER_TOL, inner_tol=INNER_TOL, mcg=MCG[mcg])
        dt = time.perf_counter() - t
        v = {"status": O.STATUS_NAMES[res.status], "outer_iters": res.outer_iters, "restarts": res.restarts,
             "inner_iters_total": res.inner_iters_total, "true_relres": res.true_relres, "seconds": round(dt, 2),
             "n": p.n, "nnz": p.nnz, "k": p.k}
        merge(key(p.name, mcg), v)
        print(r, v, flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or RECORDS)
