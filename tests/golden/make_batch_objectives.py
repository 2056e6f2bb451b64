"""Write tests/golden/batch_maxcut_objectives.json: the FP64 CPU oracle's
LOBPCG-ADMM (Algorithm 1 with the projection of Algorithm 3) objectives of a
small uneven max-cut batch, the expected values of the GPU's mixed-precision
batch test.  Calls only oracle/ and the seeded input generator.

    python tests/golden/make_batch_objectives.py
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

# the batch recipe of the batched workload (n ~ U{64..n_hi}, p ~ U[0.02, 0.2])
COUNT, N_HI = 8, 256
SETTINGS = dict(eps_abs=1e-4, rho=1.0, max_iter=5000, use_lobpcg=1)


def main():
    out = {"recipe": "paper_1912_02767_gb300.instances.workload_batch(count=%d, n_lo=64, n_hi=%d)" % (COUNT, N_HI),
           "settings": SETTINGS, "solver": "oracle.admm_solve (FP64, LOBPCG projection)", "instances": []}
    for i, inst in enumerate(gen.workload_batch(COUNT, 64, N_HI)):
        cons = oracle.Constraints(inst.n, inst.m, inst.cp, inst.ci, inst.cj, inst.cv)
        t0 = time.perf_counter()
        r = oracle.admm_solve(inst.n, inst.C, cons, inst.b, **SETTINGS)
        out["instances"].append({"index": i, "n": inst.n, "edges": int(len(inst.meta["edges"])),
                                 "status": r["status_name"], "iters": r["iters"], "obj": r["obj"],
                                 "r_prim": r["r_prim"], "r_dual": r["r_dual"]})
        print(i, inst.n, r["status_name"], r["iters"], r["obj"], "%.1f s" % (time.perf_counter() - t0), flush=True)
    with open(os.path.join(HERE, "batch_maxcut_objectives.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
