"""Write ``oracle/multilevel_study.json``: flexible-CG iteration counts to
1e-10 of the oracle with the one-level and two-level Schwarz preconditioners
and with a third, intermediate p-level added (``schwarz.
precondition_three_level``), on deformed boxes (right-hand side seed 0).

The study behind the choice of the multigrid's levels: an intermediate
order added to the two-level additive form does not reduce the iteration
count.  Test infrastructure: it runs the oracle only.

    python oracle/multilevel_study.py [nx ...]   (default 4; 6 takes ~25 min)
"""
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
from oracle import schwarz  # noqa: E402
from workloads import Box, rhs_global  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "multilevel_study.json")
CASES = [(7, 3), (9, 4)]  # (fine order N, intermediate order N_m)


def study(nx, N, Nm):
    box = Box(nx, nx, nx, N, 0.05)
    P = oracle.Problem(box)
    Pm = oracle.Problem(Box(nx, nx, nx, Nm, 0.05))
    b = P.to_local(rhs_global(box, 0))
    t = time.time()
    its = {}
    for name, pc in (("one_level", lambda r: schwarz.precondition(P, r)),
                     ("two_level", lambda r: schwarz.precondition(P, r, coarse=True)),
                     ("three_level", lambda r: schwarz.precondition_three_level(P, Pm, r))):
        _, it, rel, _ = P.fcg(b, pc, tol=1e-10, maxit=1000)
        its[name] = it
    return {"nx": nx, "N": N, "N_m": Nm, "deform": 0.05, "tol": 1e-10, **its,
            "seconds": time.time() - t}


if __name__ == "__main__":
    sizes = [int(a) for a in sys.argv[1:]] or [4]
    res = [study(nx, N, Nm) for nx in sizes for N, Nm in CASES]
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps(res, indent=1))
