"""Write tests/golden/theta500_objective.json: the FP64 CPU oracle's
LOBPCG-ADMM (Algorithm 1 with the projection of Algorithm 3) objective on the
Lovasz-theta workload n = 500, p = 0.2 (seeded), rho = 10, residual 1e-4 --
the expected value of the GPU's mixed-precision solve of that workload.
Calls only oracle/ and the seeded input generator.  Takes about twenty
minutes on one core.

    python tests/golden/make_theta500_objective.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1912_02767_gb300 import instances as gen  # noqa: E402

SETTINGS = dict(eps_abs=1e-4, rho=10.0, max_iter=20000, use_lobpcg=1)


def main():
    inst = gen.workload_theta500(0)
    cons = oracle.Constraints(inst.n, inst.m, inst.cp, inst.ci, inst.cj, inst.cv)
    t0 = time.perf_counter()
    r = oracle.admm_solve(inst.n, inst.C, cons, inst.b, **SETTINGS)
    out = {"recipe": "paper_1912_02767_gb300.instances.workload_theta500(0)", "n": inst.n, "m": inst.m,
           "settings": SETTINGS, "solver": "oracle.admm_solve (FP64, LOBPCG projection)",
           "status": r["status_name"], "iters": r["iters"], "obj": r["obj"], "r_prim": r["r_prim"],
           "r_dual": r["r_dual"], "rank": r["last_rank"], "seconds": time.perf_counter() - t0}
    with open(os.path.join(HERE, "theta500_objective.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
