"""Record the oracle's full-solve iteration counts for the benchmark workloads.

The benchmark's CPU-baseline leg times a bounded sample (the first S inner
iterations) of the oracle's solve and scales it to one full solve with the
inner-iteration total stored here.  Run:  python oracle/record_counts.py
(calls only the oracle and the input generators; takes a few minutes).
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from gen import lap2d_64_k4, lap3d_128_k10  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "full_solve_counts.json")


def main():
    rec = {}
    for make in (lap2d_64_k4, lap3d_128_k10):
        p = make()
        s = O.System.from_problem(p)
        for outer_tol, inner_tol in ((1e-10, 1e-3),):
            t = time.perf_counter()
            r = O.minres_cg(s, p.b, outer_tol=outer_tol, inner_tol=inner_tol)
            dt = time.perf_counter() - t
            rec[f"{p.name}|outer={outer_tol:g}|inner={inner_tol:g}"] = {
                "status": O.STATUS_NAMES[r.status], "outer_iters": r.outer_iters, "restarts": r.restarts,
                "inner_iters_total": r.inner_iters_total, "true_relres": r.true_relres, "seconds": round(dt, 2),
                "n": p.n, "nnz": p.nnz, "k": p.k}
            print(p.name, rec[f"{p.name}|outer={outer_tol:g}|inner={inner_tol:g}"], flush=True)
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
