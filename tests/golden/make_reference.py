"""Writes tests/golden/reference_objectives.json: FP64 oracle objectives and
statuses, solved to rel-KKT 1e-7, for the larger parity workloads.  Calls
only the oracle and the seeded generators; run from the repository root:

    python tests/golden/make_reference.py
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import lpgen  # noqa: E402
import oracle  # noqa: E402

TOL = 1e-7

CASES = {
    "sb_powerlaw_seed0": lambda: lpgen.sb_powerlaw(seed=0),
    "obbt_square_10k_seed0": lambda: lpgen.obbt_square(seed=0, m=10000, n=10000, lps=64),
}


def main():
    oracle.build()
    src = open(os.path.join(ROOT, "oracle", "pdhg_oracle.c"), "rb").read()
    out = {"tol": TOL, "oracle_sha256": hashlib.sha256(src).hexdigest(), "cases": {}}
    for name, fn in CASES.items():
        w = fn()
        t = time.time()
        r = oracle.solve(w.lp, w.specs, tol=TOL, max_iter=400000, threads=os.cpu_count() or 1, lockstep=0,
                         want_xy=False)
        out["cases"][name] = {"workload": w.name, "status": r.status.tolist(), "obj": r.obj.tolist(),
                              "iters": r.iters.tolist(), "seconds": time.time() - t}
        print(name, np.bincount(r.status), f"{time.time() - t:.1f}s", flush=True)
    with open(os.path.join(ROOT, "tests", "golden", "reference_objectives.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
