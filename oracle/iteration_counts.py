"""Write ``oracle/iteration_counts.json``: the number of FP64 Jacobi-PCG
iterations the oracle needs to reach relative residual 1e-10 on the mixed
precision workload (16^3 deformed box, N = 9, right-hand side seed 0).

The CPU baseline of the benchmark times a bounded number of oracle
iterations and scales to a full solve with this count.  Test
infrastructure: it runs the oracle only.
"""
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
from workloads import MIXED_16CUBE_N9, LEARNED_16CUBE_N7, rhs_global  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "iteration_counts.json")


def count(box, seed=0, tol=1e-10):
    P = oracle.Problem(box)
    b = P.to_local(rhs_global(box, seed))
    t = time.time()
    x, it, rel, _ = P.pcg(b, tol=tol, maxit=20000)
    return {"nx": box.nx, "ny": box.ny, "nz": box.nz, "N": box.N, "deform": box.deform,
            "seed": seed, "tol": tol, "iterations": it, "final_relres": rel,
            "true_relres": P.true_relres(b, x), "seconds": time.time() - t}


if __name__ == "__main__":
    res = {"mixed_16cube_n9": count(MIXED_16CUBE_N9), "learned_16cube_n7": count(LEARNED_16CUBE_N7)}
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps(res, indent=1))
