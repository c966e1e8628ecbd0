"""Writes tests/golden/reference_objectives.json: FP64 oracle results for the
larger parity workloads.  Calls only the oracle and the seeded generators;
run from the repository root:

    python tests/golden/make_reference.py                 # every case
    python tests/golden/make_reference.py NAME ...        # only these cases
    python tests/golden/make_reference.py --threads 4 --out PATH NAME ...
                                                          # into another file (merge with --merge)
    python tests/golden/make_reference.py --merge PATH ...  # merge such files into the golden file

Whole batches (sb_powerlaw, the 10k OBBT reduction) are solved to rel-KKT
1e-7.  The full-size batches (the 128-LP strong-branching batch on the
m=1M, n=2M matrix and the 1024-LP OBBT batch on the m=n=100k matrix) take
minutes per LP in the oracle, so a seeded subset of their LPs is stored:
each LP solved alone to rel-KKT 1e-4 (the status and the iteration count
the oracle needs at the benchmark's tolerance), and solved again to rel-KKT
1e-5 for the reference objective, both within the benchmark's cap of 100k
iterations.
"""
import argparse
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
SUBSET_MAX_ITER = 100000   # the iteration cap of the benchmark (and of the paper's OBBT runs)
SUBSET_SEED = 7
OUT = os.path.join(ROOT, "tests", "golden", "reference_objectives.json")

CASES = {
    "sb_powerlaw_seed0": lambda: lpgen.sb_powerlaw(seed=0),
    "obbt_square_10k_seed0": lambda: lpgen.obbt_square(seed=0, m=10000, n=10000, lps=64),
}
# name -> (workload, LPs in the subset, tolerance of the reference objective)
SUBSET_CASES = {
    "sb_large_seed0_subset": (lambda: lpgen.sb_large(seed=0), 8, 1e-5),
    "obbt_square_seed0_subset": (lambda: lpgen.obbt_square(seed=0), 16, 1e-5),
}


def subset_indices(num_lps: int, size: int) -> list:
    """The seeded subset of a full-size batch that the golden file covers."""
    rng = np.random.default_rng(SUBSET_SEED)
    return sorted(int(i) for i in rng.choice(num_lps, size=min(size, num_lps), replace=False))


def oracle_sha() -> str:
    src = open(os.path.join(ROOT, "oracle", "pdhg_oracle.c"), "rb").read()
    return hashlib.sha256(src).hexdigest()


def load(path):
    out = {"tol": TOL, "oracle_sha256": oracle_sha(), "cases": {}}
    if os.path.exists(path):
        old = json.load(open(path))
        if old.get("oracle_sha256") == out["oracle_sha256"]:
            out["cases"] = old.get("cases", {})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="*")
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--out", default=OUT)
    ap.add_argument("--merge", nargs="*", default=None)
    args = ap.parse_args()
    oracle.build()
    if args.merge is not None:
        out = load(OUT)
        for p in args.merge:
            part = json.load(open(p))
            assert part["oracle_sha256"] == out["oracle_sha256"], f"{p} was written by another oracle source"
            out["cases"].update(part["cases"])
        json.dump(out, open(OUT, "w"), indent=1)
        return
    out = load(args.out)
    names = set(args.names)
    for name, fn in CASES.items():
        if names and name not in names:
            continue
        w = fn()
        t = time.time()
        r = oracle.solve(w.lp, w.specs, tol=TOL, max_iter=400000, threads=args.threads, lockstep=0,
                         want_xy=False)
        out["cases"][name] = {"workload": w.name, "status": r.status.tolist(), "obj": r.obj.tolist(),
                              "iters": r.iters.tolist(), "seconds": time.time() - t}
        print(name, np.bincount(r.status), f"{time.time() - t:.1f}s", flush=True)
        json.dump(out, open(args.out, "w"), indent=1)
    for name, (fn, size, ref_tol) in SUBSET_CASES.items():
        if names and name not in names:
            continue
        w = fn()
        idx = subset_indices(len(w.specs), size)
        sp = w.specs.subset(idx)
        prep = oracle.Prepared(w.lp)
        t = time.time()
        a = prep.solve(sp, tol=SUBSET_TOL, max_iter=SUBSET_MAX_ITER, threads=args.threads, lockstep=0,
                       want_xy=False)
        t_a = time.time() - t
        print(name, "tol", SUBSET_TOL, np.bincount(a.status, minlength=5), f"{t_a:.1f}s", a.iters.tolist(),
              flush=True)
        t = time.time()
        b = prep.solve(sp, tol=ref_tol, max_iter=SUBSET_MAX_ITER, threads=args.threads, lockstep=0,
                       want_xy=False)
        t_b = time.time() - t
        print(name, "tol", ref_tol, np.bincount(b.status, minlength=5), f"{t_b:.1f}s", b.iters.tolist(), flush=True)
        out["cases"][name] = {
            "workload": w.name, "lps": idx, "subset_seed": SUBSET_SEED,
            "status": a.status.tolist(), "obj": a.obj.tolist(), "iters": a.iters.tolist(), "tol": SUBSET_TOL,
            "ref_status": b.status.tolist(), "ref_obj": b.obj.tolist(), "ref_iters": b.iters.tolist(),
            "ref_tol": ref_tol, "seconds": t_a + t_b, "threads": args.threads}
        json.dump(out, open(args.out, "w"), indent=1)
        prep.close()


if __name__ == "__main__":
    main()
