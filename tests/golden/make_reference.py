"""Writes tests/golden/reference_objectives.json: FP64 oracle results for the
larger parity workloads.  Calls only the oracle and the seeded generators;
run from the repository root:

    python tests/golden/make_reference.py            # every case
    python tests/golden/make_reference.py NAME ...   # only these cases (merged)

Whole batches (sb_powerlaw, the 10k OBBT reduction) are solved to rel-KKT
1e-7.  The full-size batches (the 128-LP strong-branching batch on the
m=1M, n=2M matrix and the 1024-LP OBBT batch on the m=n=100k matrix) take
minutes per LP in the oracle, so a seeded subset of 16 LPs is stored:
first solved alone to rel-KKT 1e-4 (the status and iteration count the
oracle needs at the benchmark's tolerance), then continued from that point
to rel-KKT 1e-6 for the reference objective.
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
SUBSET_TOL = 1e-4
SUBSET_REF_TOL = 1e-6
SUBSET_SIZE = 16
SUBSET_SEED = 7
OUT = os.path.join(ROOT, "tests", "golden", "reference_objectives.json")

CASES = {
    "sb_powerlaw_seed0": lambda: lpgen.sb_powerlaw(seed=0),
    "obbt_square_10k_seed0": lambda: lpgen.obbt_square(seed=0, m=10000, n=10000, lps=64),
}
SUBSET_CASES = {
    "sb_large_seed0_subset16": lambda: lpgen.sb_large(seed=0),
    "obbt_square_seed0_subset16": lambda: lpgen.obbt_square(seed=0),
}


def subset_indices(num_lps: int) -> list:
    """The seeded subset of a full-size batch that the golden file covers."""
    rng = np.random.default_rng(SUBSET_SEED)
    return sorted(int(i) for i in rng.choice(num_lps, size=min(SUBSET_SIZE, num_lps), replace=False))


def oracle_sha() -> str:
    src = open(os.path.join(ROOT, "oracle", "pdhg_oracle.c"), "rb").read()
    return hashlib.sha256(src).hexdigest()


def main(names):
    oracle.build()
    threads = os.cpu_count() or 1
    out = {"tol": TOL, "oracle_sha256": oracle_sha(), "cases": {}}
    if os.path.exists(OUT):
        old = json.load(open(OUT))
        if old.get("oracle_sha256") == out["oracle_sha256"]:
            out["cases"] = old.get("cases", {})
    for name, fn in CASES.items():
        if names and name not in names:
            continue
        w = fn()
        t = time.time()
        r = oracle.solve(w.lp, w.specs, tol=TOL, max_iter=400000, threads=threads, lockstep=0, want_xy=False)
        out["cases"][name] = {"workload": w.name, "status": r.status.tolist(), "obj": r.obj.tolist(),
                              "iters": r.iters.tolist(), "seconds": time.time() - t}
        print(name, np.bincount(r.status), f"{time.time() - t:.1f}s", flush=True)
        json.dump(out, open(OUT, "w"), indent=1)
    for name, fn in SUBSET_CASES.items():
        if names and name not in names:
            continue
        w = fn()
        idx = subset_indices(len(w.specs))
        sp = w.specs.subset(idx)
        prep = oracle.Prepared(w.lp)
        t = time.time()
        a = prep.solve(sp, tol=SUBSET_TOL, max_iter=200000, threads=threads, lockstep=0, want_xy=True)
        t_a = time.time() - t
        print(name, "tol", SUBSET_TOL, np.bincount(a.status, minlength=5), f"{t_a:.1f}s", a.iters.tolist(),
              flush=True)
        t = time.time()
        b = prep.solve(sp, tol=SUBSET_REF_TOL, max_iter=200000, threads=threads, lockstep=0, want_xy=False,
                       warm_x=a.x, warm_y=a.y)
        t_b = time.time() - t
        print(name, "tol", SUBSET_REF_TOL, np.bincount(b.status, minlength=5), f"{t_b:.1f}s", flush=True)
        out["cases"][name] = {
            "workload": w.name, "lps": idx, "subset_seed": SUBSET_SEED,
            "status": a.status.tolist(), "obj": a.obj.tolist(), "iters": a.iters.tolist(), "tol": SUBSET_TOL,
            "ref_status": b.status.tolist(), "ref_obj": b.obj.tolist(), "ref_iters": b.iters.tolist(),
            "ref_tol": SUBSET_REF_TOL, "seconds": t_a + t_b, "threads": threads}
        json.dump(out, open(OUT, "w"), indent=1)
        prep.close()


if __name__ == "__main__":
    main(set(sys.argv[1:]))
