"""Benchmark: LPs solved per second by the batched PDHG solver on one GB300.

A step is one complete batched solve (every LP of the batch to rel-KKT 1e-4,
all hot-path steps: both fused SpMM steps, the KKT checks, restarts,
compaction) of a seeded synthetic batch whose matrix is already resident on
the GPU.  The default workload is the large strong-branching batch: 128
children of a shared A with m=1M, n=2M, nnz ~10.5M (rows of 3-8 nonzeros
plus 500 dense rows of 10k), FP32 iterates with double-float (about 48-bit)
KKT and restart checks; its iterate blocks (1 GB per block) exceed L2 many
times over.  The 1024-LP bound-tightening batch (m=n=100k, nnz=1M) is timed
once more as an extra key.

Prints ONE JSON line (rank 0).  Under torchrun with N>1 every rank solves
its own, independently seeded batch (weak scaling, no collective on the data
path); value = LPs solved by all ranks / max-over-ranks time.

--impl reference times the CPU oracle (plain FP64 C, all host cores) on a
bounded sample of the same workload; it is the slow reference arm.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lpgen  # noqa: E402

METRIC = "LPs solved/s to rel-KKT 1e-4 (batched vs B=1 loop); SpMM HBM GB/s; p99 lat"
UNIT = "LPs/s"
TOL = 1e-4
FALLBACK_HBM_GBS = 6800.0

# cpu_lps: the oracle's default sample of whole solves; golden: the seeded
# subset of a full-size batch whose oracle results (iterations to 1e-4 and
# reference objectives) tests/golden/make_reference.py stores, for workloads
# where one oracle solve takes minutes: there the oracle's sample is a bounded
# number of iterations, scaled by its own iteration counts
WORKLOADS = {
    "sb_powerlaw": dict(fn=lambda seed: lpgen.sb_powerlaw(seed=seed), max_iter=100000, cpu_lps=64,
                        golden="sb_powerlaw_seed0"),
    "sb_small": dict(fn=lambda seed: lpgen.sb_small(seed=seed), max_iter=100000, cpu_lps=16, golden=None),
    "obbt_square": dict(fn=lambda seed: lpgen.obbt_square(seed=seed), max_iter=100000, cpu_lps=0,
                        golden="obbt_square_seed0_subset"),
    "sb_large": dict(fn=lambda seed: lpgen.sb_large(seed=seed), max_iter=100000, cpu_lps=0,
                     golden="sb_large_seed0_subset"),
}
DTYPE_MIXED = "f32-iterates/double-float-checks"
# iterations of the oracle's bounded sample (per LP) where whole solves take minutes
ORACLE_SAMPLE_ITERS = 64


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def golden_case(name):
    """The oracle's stored results for `name`, or None when the file is
    missing, lacks the case, or was written by another oracle source."""
    if not name:
        return None
    try:
        g = json.load(open(os.path.join(ROOT, "tests", "golden", "reference_objectives.json")))
        src = open(os.path.join(ROOT, "oracle", "pdhg_oracle.c"), "rb").read()
        if g.get("oracle_sha256") != hashlib.sha256(src).hexdigest():
            return None
        return g["cases"].get(name)
    except Exception:
        return None


def golden_lps_and_ref(name, q):
    """(LP indices, oracle status at the solve tolerance, reference objective)
    of the stored case: a seeded subset, or the whole batch."""
    c = golden_case(name)
    if c is None:
        return None
    if "lps" in c:
        return list(c["lps"]), np.asarray(c["status"]), np.asarray(c["ref_obj"]), np.asarray(c["iters"])
    return list(range(q)), np.asarray(c["status"]), np.asarray(c["obj"]), None


def golden_ref_tol(name):
    c = golden_case(name)
    if c is None:
        return None
    return c.get("ref_tol", c.get("tol"))


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_workload(name: str, seed: int, rank: int):
    """Weak scaling over replicas: rank r solves its own batch, seeded seed + r,
    so ranks share no data and need no collective on the data path."""
    return WORKLOADS[name]["fn"](seed + rank)


def reduce_over_ranks(dist, elapsed, solved, device):
    """Whole-job figures over the replicas: the slowest rank's time (max) and
    the LPs solved by all ranks (sum).  dist is torch.distributed or None."""
    if dist is None:
        return float(elapsed), int(solved)
    import torch

    t = torch.tensor([float(elapsed)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(solved)], device=device, dtype=torch.float64)
    dist.all_reduce(c)
    return float(t.item()), int(round(c.item()))


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def solved(res) -> int:
    st = res["status"]
    return int(np.sum((st == 0) | (st == 1) | (st == 2)))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"lpb_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def step_source_sha(csrc: str) -> str:
    """Hash of the step kernels' source: their device code (lpb_step.h),
    their launches (lpb_iter.cu) and the long-row segments they take
    (lpb_internal.h, lpb_setup.cu)."""
    h = hashlib.sha256()
    for f in ("lpb_step.h", "lpb_iter.cu", "lpb_internal.h", "lpb_setup.cu"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_name: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary and how they were
    taken, if they were taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except Exception:
        return None, None
    csrc = os.path.join(ROOT, "paper_2601_21990_gb300", "csrc")
    h = step_source_sha(csrc)
    ent = d.get(workload, {}).get(kernel_name)
    if not ent or ent.get("step_source_sha") != h:
        return None, None
    return ent.get("dram_bytes_per_launch"), f"ncu DRAM bytes of one {ent.get('ncol')}-LP launch: {ent.get('note')}"


def oracle_scaled_sample(w, gold, cores, iters):
    """The oracle on the stored subset for `iters` iterations per LP (OpenMP
    over LPs, the set-up done once outside the timing): per LP-iteration core
    time, and the wall time the subset's whole solve takes at that rate with
    the oracle's own iteration counts to 1e-4 (the longest LP, or the total
    over the cores, whichever is larger)."""
    import oracle

    oracle.build()
    lps, status, _, need = gold
    sp = w.specs.subset(lps)
    t = time.perf_counter()
    prep = oracle.Prepared(w.lp)
    setup_s = time.perf_counter() - t
    return prep, sp, setup_s, status, need


def oracle_sample_rate(prep, sp, status, need, cores, iters):
    s = len(sp)
    t = time.perf_counter()
    prep.solve(sp, tol=TOL, max_iter=iters, threads=cores, lockstep=0, want_xy=False)
    dt = time.perf_counter() - t
    par = max(1, min(cores, s))
    per_lp_iter = dt * par / (iters * s)  # core-seconds of one LP-iteration
    wall = max(float(np.max(need)), float(np.sum(need)) / par) * per_lp_iter
    solved = int(np.sum(status <= 2))
    return solved / wall, dt, wall


def run_reference(args, rank, world):
    """The CPU oracle, as it stands, on the host cores: a bounded sample."""
    if world > 1 and rank != 0:
        return
    import oracle

    oracle.build()
    w = WORKLOADS[args.workload]["fn"](args.seed)
    q = len(w.specs)
    cores = os.cpu_count() or 1
    max_iter = WORKLOADS[args.workload]["max_iter"]
    gold = golden_lps_and_ref(WORKLOADS[args.workload]["golden"], q)
    if WORKLOADS[args.workload]["cpu_lps"] == 0:
        if gold is None or gold[3] is None:
            print(json.dumps({"impl": "reference", "unavailable": "one oracle solve of this workload takes minutes "
                              "and the stored oracle iteration counts are missing or stale"}), flush=True)
            return
        prep, sp, setup_s, status, need = oracle_scaled_sample(w, gold, cores, ORACLE_SAMPLE_ITERS)
        iters = max(4, ORACLE_SAMPLE_ITERS // 4)
        for _ in range(args.warmup if args.ref_warmup else 0):
            oracle_sample_rate(prep, sp, status, need, cores, iters)
        times, walls = [], []
        for _ in range(args.steps):
            _, dt, wall = oracle_sample_rate(prep, sp, status, need, cores, iters)
            times.append(dt)
            walls.append(wall)
        solved = int(np.sum(status <= 2))
        v = solved / float(np.mean(walls))
        desc = (f"{len(sp)} of {q} LPs of {w.name} (the stored seeded subset), each alone, OpenMP over LPs, "
                f"{iters} iterations per LP per step; LPs/s = LPs the oracle solves at 1e-4 / the time its own "
                f"iteration counts to 1e-4 take at the measured rate; set-up {setup_s:.1f} s once, not timed")
        ms = 1e3 * float(np.mean(walls))
        sample_lps = len(sp)
    else:
        # a bounded sample per step: about 640 LP solves over the whole run
        sample = min(q, args.ref_lps, max(4, 640 // max(args.steps, 1)))
        sp = w.specs.subset(range(sample))
        prep = oracle.Prepared(w.lp)
        for _ in range(args.warmup if args.ref_warmup else 0):
            prep.solve(sp, tol=TOL, max_iter=max_iter, threads=cores, lockstep=0, want_xy=False)
        times, nsolved = [], 0
        for _ in range(args.steps):
            t = time.perf_counter()
            r = prep.solve(sp, tol=TOL, max_iter=max_iter, threads=cores, lockstep=0, want_xy=False)
            times.append(time.perf_counter() - t)
            nsolved += int(np.sum(r.status <= 2))
        total = sum(times)
        v = nsolved / total
        desc = f"{sample} of {q} LPs of {w.name}, each solved alone (own restarts), OpenMP over LPs"
        ms = 1e3 * total / args.steps
        sample_lps = sample
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "tol": TOL, "sample_lps": sample_lps},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "cpu": cpu_model(), "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def cpu_baseline(w, name, cores, budget_lps):
    import oracle

    oracle.build()
    q = len(w.specs)
    if budget_lps <= 0:
        gold = golden_lps_and_ref(WORKLOADS[name]["golden"], q)
        if gold is None or gold[3] is None:
            return {"value": None, "unit": UNIT, "cores": cores, "cpu": cpu_model(), "kind": "oracle",
                    "sample": "none: one oracle solve takes minutes and the stored iteration counts are missing"}
        prep, sp, setup_s, status, need = oracle_scaled_sample(w, gold, cores, ORACLE_SAMPLE_ITERS)
        v, dt, wall = oracle_sample_rate(prep, sp, status, need, cores, ORACLE_SAMPLE_ITERS)
        prep.close()
        return {"value": v, "unit": UNIT, "cores": cores, "cpu": cpu_model(), "kind": "oracle",
                "sample": f"{len(sp)} of {q} LPs of {w.name} (the stored seeded subset), each alone, OpenMP over "
                          f"LPs, {ORACLE_SAMPLE_ITERS} iterations per LP in {dt:.1f} s; LPs/s = LPs the oracle "
                          f"solves at 1e-4 / the {wall:.0f} s its own iteration counts to 1e-4 "
                          f"(max {int(np.max(need))}) take at that rate; set-up {setup_s:.1f} s, not counted",
                "setup_s": setup_s}
    sample = min(q, budget_lps)
    sp = w.specs.subset(range(sample))
    t = time.perf_counter()
    r = oracle.solve(w.lp, sp, tol=TOL, max_iter=100000, threads=cores, lockstep=0, want_xy=False)
    dt = time.perf_counter() - t
    # the B=1 loop on one core, on a smaller sample
    one = min(q, 2)
    t = time.perf_counter()
    r1 = oracle.solve(w.lp, w.specs.subset(range(one)), tol=TOL, max_iter=100000, threads=1, lockstep=0,
                      want_xy=False)
    dt1 = time.perf_counter() - t
    return {"value": int(np.sum(r.status <= 2)) / dt, "unit": UNIT, "cores": cores, "cpu": cpu_model(),
            "kind": "oracle",
            "sample": f"{sample} of {q} LPs of {w.name}, each alone, OpenMP over LPs, {dt:.1f} s",
            "single_thread_b1": {"value": int(np.sum(r1.status <= 2)) / dt1, "unit": UNIT, "cores": 1,
                                 "sample": f"{one} LPs one after another on one core, {dt1:.1f} s"}}


def oracle_error(w, name, batch, res):
    """Error of this run's results against the FP64 oracle, on the LPs the
    oracle has stored results for: status agreement, the largest relative
    objective error against the oracle's reference objective, and the largest
    relative KKT residual of the returned (x, y) in the oracle's evaluation."""
    import oracle

    q = len(w.specs)
    gold = golden_lps_and_ref(WORKLOADS[name]["golden"], q) if name in WORKLOADS else None
    if gold is None:
        return {"unavailable": "no stored oracle results for this workload and oracle source"}
    lps, status, ref_obj, _ = gold
    st = res["status"][lps]
    both = (status == 0) & (st == 0)
    err = np.abs(res["obj"][lps][both] - ref_obj[both]) / (1.0 + np.abs(ref_obj[both]))
    kkt = []
    for i, lp_i in enumerate(lps[:16]):
        if st[i] != 0:
            continue
        r, x, y = batch.result(int(lp_i))
        k = oracle.kkt_spec(w.lp, w.specs, int(lp_i), x, y)
        kkt.append(max(k["rel_primal"], k["rel_dual"], k["rel_gap"]))
    return {"lps": len(lps), "status_equal": int(np.sum(st == status)),
            "max_rel_obj_err": float(err.max()) if err.size else None,
            "max_oracle_rel_kkt": float(max(kkt)) if kkt else None, "kkt_lps": len(kkt),
            "ref_tol": golden_ref_tol(WORKLOADS[name]["golden"]),
            "what": "against the FP64 oracle: statuses at this tolerance, reference objectives solved to ref_tol "
                    "(or 1e-7 for whole batches), and the oracle's own KKT evaluation of the returned points, on "
                    "the stored LPs of this batch"}


def run_serving(args, rank, world, local):
    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist_mod.init_process_group("nccl")
        dist = dist_mod
    line = serving_measure(args, rank, world, local, dist, args.requests, args.warmup)
    if line is not None:
        print(json.dumps(line), flush=True)


def serving_measure(args, rank, world, local, dist, requests, warmup):
    """Continuous batching over five matrices (m = 1k .. 200k, n = 2m, power-
    law rows): first the capacity with every request queued at once, then a
    seeded Poisson stream at args.load of that capacity; latency is each
    request's submit-to-done time.  Every request warm-starts from its
    matrix's base LP, solved first and kept on the device.  Returns the
    bench line on rank 0 (None elsewhere)."""
    import torch

    from paper_2601_21990_gb300 import lpb

    mats = lpgen.serving_matrices(seed0=args.seed + 10 * rank)
    # smaller matrices get more urgent streams: their short intervals take SMs
    # ahead of the large matrices' queued kernels
    order = np.argsort([lp.m for lp in mats])
    prio = {int(k): -(len(mats) - 1 - r) if args.priorities else 0 for r, k in enumerate(order)}
    handles = [lpb.Handle(lp, precision=lpb.MIXED, device=local, stream_priority=prio[k])
               for k, lp in enumerate(mats)]
    srv = lpb.Server(lane_columns=512, polish_columns=64, max_groups=64, device=local)
    mids = [srv.attach(h) for h in handles]
    parents = [srv.submit(mid, lpb.specs_array([0], [-1]), tol=TOL, max_iter=100000) for mid in mids]
    for p in parents:
        srv.wait(p)
    specs_np = {}

    def submit(k, sp):
        key = id(sp)
        if key not in specs_np:
            specs_np[key] = lpb.specs_from(sp)
        return srv.submit(mids[k], specs_np[key], tol=TOL, max_iter=100000, warm_request=parents[k], warm_lp=0)

    def drain(ids):
        solved, d2h = 0, 0
        for r in ids:
            srv.wait(r)
            res = srv.results(r)
            d2h += res.nbytes
            solved += solved_count(res)
        return solved, d2h

    warm = lpgen.serving_stream(mats, seed=99, count=max(warmup, 1) * 5)
    for r in [submit(k, sp) for _, k, sp in warm]:
        srv.wait(r)
        srv.release(r)
    # capacity: everything queued at once; the rate while 80% of the LPs
    # finish (the last few requests alone would measure their latency)
    cap_stream = lpgen.serving_stream(mats, seed=101, count=max(requests // 2, 10))
    cap_ids = [submit(k, sp) for _, k, sp in cap_stream]
    done = []
    for r in cap_ids:
        srv.wait(r)
        info = srv.info(r)
        done.append((info.t_done, info.t_submit, solved_count(srv.results(r))))
        srv.release(r)
    t_first = min(d[1] for d in done)
    done.sort()
    tot = sum(d[2] for d in done)
    acc, cap = 0, None
    for t_d, _, c in done:
        acc += c
        if acc >= 0.8 * tot:
            cap = acc / max(t_d - t_first, 1e-9)
            break
    stream = lpgen.serving_stream(mats, seed=100, count=requests)
    mean_lps = float(np.mean([len(sp) for _, _, sp in stream]))
    rate = args.load * cap / mean_lps  # requests per second
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    st0 = srv.stats()
    ids, t_sub = [], []
    t0 = time.perf_counter()
    t_next = t0
    h2d = 0
    for gap, k, sp in stream:
        t_next += gap / rate
        dt = t_next - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        ids.append(submit(k, sp))
        h2d += specs_np[id(sp)].nbytes
    nsolved, d2h = drain(ids)
    wall = time.perf_counter() - t0
    torch.cuda.synchronize()
    clk = clocks.stop()
    st1 = srv.stats()
    lat, per_mat = [], {}
    for (gap, k, sp), r in zip(stream, ids):
        info = srv.info(r)
        lat.append(1e3 * (info.t_done - info.t_submit))
        per_mat.setdefault(k, []).append((lat[-1], 1e3 * (info.t_admit - info.t_submit), info.iters,
                                          info.polished))
        srv.release(r)
    total_s = wall
    total_s, nsolved_all = reduce_over_ranks(dist, wall, nsolved, f"cuda:{local}")
    value = nsolved_all / total_s
    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": 1, "warmup": warmup,
            "ms_per_step": 1e3 * total_s, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE_MIXED, "data": "synthetic",
            "config": {"workload": "serving: 5 power-law matrices m=1k..200k n=2m, Poisson requests of U{1..256} "
                                   "strong-branching children, warm start from the parent LP on the device",
                       "requests": len(ids), "lps": int(sum(len(sp) for _, _, sp in stream)), "tol": TOL,
                       "load": args.load, "capacity_lps_per_s": cap, "rate_req_per_s": rate,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "inputs (200k-row matrix lanes) exceed L2"},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(np.max(lat)), "what": "request submit to done"},
            "latency_by_matrix": {f"m={mats[k].m}": {
                "requests": len(v), "p50_ms": float(np.percentile([a[0] for a in v], 50)),
                "p99_ms": float(np.percentile([a[0] for a in v], 99)),
                "queue_p50_ms": float(np.percentile([a[1] for a in v], 50)),
                "iters_p50": float(np.percentile([a[2] for a in v], 50)),
                "polished": int(sum(a[3] for a in v))} for k, v in sorted(per_mat.items())},
            "server": {"intervals": st1.intervals - st0.intervals,
                       "admitted_while_busy": st1.admitted_while_busy - st0.admitted_while_busy,
                       "migrations": st1.migrations - st0.migrations,
                       "column_iters": st1.column_iters - st0.column_iters,
                       "busy_frac": (st1.busy_s - st0.busy_s) / wall},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "what": "the serving API itself: host records in, host results out"},
            "gpu_launches": int(st1.kernels - st0.kernels),
            "clocks": clk,
        }
    srv.close()
    return line


def cusparse_spmm(lp, ncol, dev, reps=20):
    """The paper's SpMM engine on the dual step's shape: cuSPARSE CSR SpMM
    (torch.sparse.mm) of A (FP32 values) by a dense n x ncol FP32 block, no
    epilogue; microseconds per product and algorithmic GB/s (A's values and
    indices, the dense block read once, the m x ncol product written)."""
    import torch

    a = torch.sparse_csr_tensor(torch.tensor(lp.row_ptr, dtype=torch.int32), torch.tensor(lp.col_idx),
                                torch.tensor(lp.vals, dtype=torch.float32), size=(lp.m, lp.n)).to(dev)
    x = torch.randn(lp.n, ncol, device=dev)
    for _ in range(3):
        y = torch.sparse.mm(a, x)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        y = torch.sparse.mm(a, x)
    e1.record()
    torch.cuda.synchronize()
    us = 1e3 * e0.elapsed_time(e1) / reps
    by = 8.0 * lp.nnz + 4.0 * (lp.m + 1) + 4.0 * ncol * (lp.n + lp.m)
    del y
    return {"us": us, "GBps": by / (us * 1e-6) / 1e9, "what": f"torch.sparse.mm (cuSPARSE) A @ X, X {lp.n}x{ncol} FP32"}


def solved_count(res) -> int:
    st = res["status"]
    return int(np.sum((st == 0) | (st == 1) | (st == 2)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sb_large", choices=sorted(WORKLOADS) + ["serving", "joint"])
    ap.add_argument("--extra-obbt", type=int, default=1,
                    help="also time the 1024-LP bound-tightening batch once (an extra key)")
    ap.add_argument("--extra-joint", type=int, default=1,
                    help="also time eight small matrices solved alone and as one joint solve (an extra key)")
    ap.add_argument("--extra-serving", type=int, default=80,
                    help="also run the serving workload with this many requests (an extra key; 0: skip)")
    ap.add_argument("--requests", type=int, default=160, help="serving: requests in the timed Poisson stream")
    ap.add_argument("--load", type=float, default=0.7, help="serving: arrival rate as a fraction of capacity")
    ap.add_argument("--priorities", type=int, default=1, help="serving: stream priorities by matrix size")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--ref-lps", type=int, default=64)
    ap.add_argument("--ref-warmup", action="store_true")
    ap.add_argument("--cpu-lps", type=int, default=-1,
                    help="oracle sample size for cpu_baseline (-1: the workload's default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--b1-lps", type=int, default=8, help="LPs solved one at a time for the B=1 comparison")
    ap.add_argument("--lps", type=int, default=0, help="solve only the first N LPs of the workload (0: all)")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the timed solves and one profiled repeat: no B=1 loop, cuSPARSE comparison, width "
                         "sweep or end-to-end leg (the form the ncu captures run)")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        if args.workload in ("serving", "joint"):
            print(json.dumps({"impl": "reference", "unavailable": "the oracle has no serving loop or joint solve; "
                              "the reference arm runs on the batch workloads"}), flush=True)
            return
        run_reference(args, rank, world)
        return
    if args.workload == "serving":
        run_serving(args, rank, world, local)
        return
    if args.workload == "joint":
        # the joint-solve comparison alone (its key of the default line)
        import torch

        from paper_2601_21990_gb300 import lpb

        torch.cuda.set_device(local)
        if rank == 0:
            print(json.dumps({"workload": "joint", "joint_solve": joint_extra(lpb, torch, args.seed)}), flush=True)
        return

    import torch

    from paper_2601_21990_gb300 import lpb

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist_mod.init_process_group("nccl")
        dist = dist_mod
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    # each rank: its own seeded batch (weak scaling)
    w = rank_workload(args.workload, args.seed, rank)
    if args.lps > 0 and args.lps < len(w.specs):
        w = lpgen.Workload(w.lp, w.specs.subset(range(args.lps)), w.precision, f"{w.name} (first {args.lps} LPs)")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    clocks = ClockSampler(local)
    m = measure(args, lpb, torch, w, args.workload, dev, stream, flush, args.steps, args.warmup, dist, clocks,
                extras=not args.no_extras, check_oracle=rank == 0 and world == 1 and args.lps == 0)

    # the 1024-LP bound-tightening batch (m = n = 100k, nnz = 1M), once more
    # as an extra key: one timed solve, its own roofline and oracle error
    extra = None
    if args.extra_obbt and args.workload != "obbt_square" and not args.no_extras:
        wo = rank_workload("obbt_square", args.seed, rank)
        mo = measure(args, lpb, torch, wo, "obbt_square", dev, stream, flush, 1, 0, dist, None, extras=False,
                     check_oracle=rank == 0 and world == 1)
        extra = {"workload": wo.name, "m": wo.lp.m, "n": wo.lp.n, "nnz": wo.lp.nnz, "lps_per_step": len(wo.specs),
                 "value": mo["value"], "unit": UNIT, "ms_per_step": mo["ms_per_step"], "steps": 1,
                 "lps_solved_per_step": mo["lps_solved_per_step"], "roofline": mo["roofline"],
                 "time_split_ms_per_step": mo["time_split_ms_per_step"], "oracle_error": mo["oracle_error"],
                 "polish": mo["polish"], "gpu_launches": mo["gpu_launches"]}
        if rank == 0 and not args.no_cpu_baseline and world == 1:
            extra["cpu_baseline"] = cpu_baseline(wo, "obbt_square", os.cpu_count() or 1, 0)

    joint = None
    if args.extra_joint and not args.no_extras and rank == 0:
        joint = joint_extra(lpb, torch, args.seed)
    # continuous batching (the serving workload), shortened: p50 / p99 latency
    serving = None
    if args.extra_serving > 0 and not args.no_extras and rank == 0 and world == 1:
        sl = serving_measure(args, 0, 1, local, None, args.extra_serving, 3)
        serving = {k: sl[k] for k in ("value", "unit", "ms_per_step", "config", "latency_ms", "latency_by_matrix",
                                      "server", "e2e", "gpu_launches", "clocks")}

    out = None
    if rank == 0:
        cores = os.cpu_count() or 1
        cpu_lps = args.cpu_lps if args.cpu_lps >= 0 else WORKLOADS[args.workload]["cpu_lps"]
        cpu = None if args.no_cpu_baseline or world > 1 else cpu_baseline(w, args.workload, cores, cpu_lps)
        lp = w.lp
        out = {
            "metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": m["dtype"], "data": "synthetic",
            "config": {"workload": w.name, "m": lp.m, "n": lp.n, "nnz": lp.nnz, "lps_per_step": len(w.specs),
                       "tol": TOL, "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (1 GB iterate blocks) and L2 flushed between steps (256 MB "
                             "write)" if lp.n * len(w.specs) * 4 > 256e6 else "flushed between steps (256 MB write)",
                       "lps_solved_per_step": m["lps_solved_per_step"]},
            "roofline": m["roofline"],
            "time_split_ms_per_step": m["time_split_ms_per_step"],
            "oracle_error": m["oracle_error"],
            "cusparse_dual_spmm": m.get("cusparse"),
            "width_sweep": m.get("width_sweep"),
            "b1_loop": m.get("b1_loop"),
            "latency_ms": m["latency_ms"],
            "cpu_baseline": cpu,
            "e2e": m.get("e2e"),
            "gpu_launches": m["gpu_launches"],
            "setup_ms": m["setup_ms"],
            "polish": m["polish"],
            "obbt_square": extra,
            "joint_solve": joint,
            "serving": serving,
            "clocks": m["clocks"],
        }
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)


JOINT_ROWS = (1000, 1250, 1500, 1750, 2000, 2250, 2500, 2750)
JOINT_LPS = 32


def joint_extra(lpb, torch, seed, reps=3):
    """Eight small strong-branching matrices (power-law rows as sb_powerlaw,
    m = 1000 .. 2750, n = 2m), 32 LPs each: solved one matrix after another
    and as one joint solve (lpb_solve_multi: one primal and one dual step
    launch per iteration for all eight).  LPs/s of both (best of two rounds
    of `reps` solves each) and whether the joint results equal the alone
    ones bitwise."""
    mats = lpgen.serving_matrices(seed0=seed + 10, rows=JOINT_ROWS)
    rng = np.random.default_rng(seed + 5)
    specs = [lpgen.sb_specs(lp.x0, rng.choice(lp.n, size=JOINT_LPS // 2, replace=False)) for lp in mats]
    hs = [lpb.Handle(lp, precision=lpb.MIXED) for lp in mats]
    alone = lambda: [h.solve(sp, tol=TOL, max_iter=100000) for h, sp in zip(hs, specs)]
    joint = lambda: lpb.Handle.solve_multi(hs, specs, tol=TOL, max_iter=100000)
    ra, rj = alone(), joint()
    same = all(np.array_equal(a.results(), j.results()) for a, j in zip(ra, rj))
    best = {}
    for _ in range(2):
        for nm, f in (("alone", alone), ("joint", joint)):
            torch.cuda.synchronize()
            t = time.perf_counter()
            for _ in range(reps):
                bs = f()
            torch.cuda.synchronize()
            best[nm] = min(best.get(nm, 1e30), (time.perf_counter() - t) / reps)
    # one more joint solve inside the NVTX range the ncu captures select
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")
    joint()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    lps = JOINT_LPS * len(mats)
    solved = sum(int(np.sum(b.results()["status"] <= 2)) for b in bs)
    return {"workload": f"{len(mats)} power-law SB matrices m={JOINT_ROWS[0]}..{JOINT_ROWS[-1]} n=2m, "
                        f"{JOINT_LPS} LPs each, fp32-iterates/double-float-checks",
            "lps": lps, "lps_solved": solved, "unit": UNIT,
            "alone": {"value": solved / best["alone"], "ms": best["alone"] * 1e3,
                      "step_launches_per_iteration": 2 * len(mats)},
            "joint": {"value": solved / best["joint"], "ms": best["joint"] * 1e3, "step_launches_per_iteration": 2},
            "speedup": best["alone"] / best["joint"], "bitwise_equal_to_alone": bool(same),
            "timing": "wall clock of complete solves (host API, device-resident specs excluded), synchronized"}


def measure(args, lpb, torch, w, name, dev, stream, flush, steps, warmup, dist, clocks, extras, check_oracle):
    """Timed batched solves of workload w (graphs + programmatic dependent
    launch, device-resident inputs), then one profiled repeat with events
    around every launch for the roofline, the oracle error of one batch, and
    (extras) the cuSPARSE comparison, width sweep, B=1 loop and end-to-end
    leg through the host API."""
    world = dist.get_world_size() if dist else 1
    local = dev.index
    max_iter = WORKLOADS[name]["max_iter"]
    precision = lpb.FP64 if w.precision == "fp64" else lpb.MIXED
    # timed solves: CUDA graphs and programmatic dependent launch, no per-launch events
    opts = lpb.lpb_default_options(precision=precision, profile=0, device=local, cuda_stream=stream.cuda_stream)
    h = lpb.Handle(w.lp, options=opts)
    specs_np = lpb.specs_from(w.specs)
    specs_dev = torch.from_numpy(specs_np.view(np.uint8).copy()).to(dev)
    q = len(w.specs)

    def one_step():
        b = h.solve_dev(specs_dev, tol=TOL, max_iter=max_iter)
        res = b.results()
        prof = b.profile()
        b.free()
        return res, prof

    for _ in range(warmup):
        one_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    nsolved, profs = 0, []
    torch.cuda.nvtx.range_push("timed")
    for k in range(steps):
        flush.zero_()  # L2 (129 MB) flushed between timed solves
        ev[k][0].record(stream)
        res, prof = one_step()
        ev[k][1].record(stream)
        nsolved += solved(res)
        profs.append(prof)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop() if clocks else None
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    gpu_launches = int(sum(p.kernels for p in profs))
    switch_iters = [int(p.fp64_switch_iter) for p in profs]
    # per-launch kernel times: the same solve again with CUDA events around
    # every launch (plain launches; graphs and PDL need no events between kernels)
    hp = lpb.Handle(w.lp, options=lpb.lpb_default_options(precision=precision, profile=1, device=local,
                                                         cuda_stream=stream.cuda_stream))
    prof_steps = 1 if not extras else max(1, min(steps, 3))
    pprofs = []
    kept = None
    for i in range(prof_steps):
        flush.zero_()
        b = hp.solve_dev(specs_dev, tol=TOL, max_iter=max_iter)
        pprofs.append(b.profile())
        if i == 0 and check_oracle:
            kept = b
        else:
            b.free()
    # the oracle's evaluation of one batch's results (the same LPs, bitwise the
    # same results as the timed solves: graphs and PDL do not change them)
    oerr = None
    if check_oracle:
        oerr = oracle_error(w, name, kept, kept.results())
        kept.free()
    hp.close()
    total_ms, nsolved_all = reduce_over_ranks(dist, total_ms, nsolved, dev)
    value = nsolved_all / (total_ms / 1e3)

    # roofline of the dominant kernel, from the library's CUDA events on this stream
    ms = np.array([[p.ms[i] for i in range(4)] for p in pprofs]).sum(0)
    by = np.array([[p.bytes[i] for i in range(4)] for p in pprofs]).sum(0)
    la = np.array([[p.launches[i] for i in range(4)] for p in pprofs]).sum(0)
    names = ["k_primal (A~^T Y + primal step)", "k_dual (A~ Xbar + dual step)"]
    dom = int(np.argmax(ms[:2]))
    achieved = by[dom] / (ms[dom] / 1e3) / 1e9
    peak, peak_kind = measured_peak()
    traffic, traffic_note = ncu_traffic(["k_primal", "k_dual"][dom], name)
    other = 1 - dom
    out = {
        "value": value, "ms_per_step": total_ms / steps, "lps_solved_per_step": nsolved / steps,
        "dtype": "f64" if precision == lpb.FP64 else DTYPE_MIXED,
        "roofline": {"bound": "hbm", "kernel": names[dom], "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                     "traffic": traffic, "traffic_note": traffic_note, "launches": int(la[dom]),
                     "avg_launch_us": 1e3 * ms[dom] / max(la[dom], 1),
                     "timing": f"CUDA events around every launch over {prof_steps} profiled repeat(s) of the "
                               "timed solve (plain launches)",
                     "other_kernel": {"kernel": names[other], "achieved": by[other] / (ms[other] / 1e3) / 1e9
                                      if ms[other] > 0 else None,
                                      "frac": by[other] / (ms[other] / 1e3) / 1e9 / peak if ms[other] > 0 else None,
                                      "avg_launch_us": 1e3 * ms[other] / max(la[other], 1)}},
        "time_split_ms_per_step": {"primal_step": ms[0] / prof_steps, "dual_step": ms[1] / prof_steps,
                                   "check_spmm": ms[2] / prof_steps, "check_reduce": ms[3] / prof_steps,
                                   "what": "profiled repeats (plain launches, events around each)"},
        "oracle_error": oerr,
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                       "what": "one batched solve"},
        "gpu_launches": gpu_launches,
        "setup_ms": pprofs[0].setup_ms if pprofs else None,
        "polish": {"arith": "dfloat" if opts.polish_arith == lpb.POLISH_DFLOAT else "fp64",
                   "switch_iter_per_step": switch_iters},
        "clocks": clk,
    }
    if not extras:
        h.close()
        return out

    # the paper's engine on the same shape, and the step time against the batch
    # width (the synthetic analogue of the paper's SpMM-vs-N figure)
    try:
        out["cusparse"] = cusparse_spmm(w.lp, q, dev)
    except Exception as ex:  # torch without CSR SpMM support on this device
        out["cusparse"] = {"unavailable": str(ex)[:120]}
    # widths whose lane and check workspace fit in half the free memory
    # (about 44 n + 36 m bytes per FP32 column)
    per_col = 44.0 * w.lp.n + 36.0 * w.lp.m
    free_b = torch.cuda.mem_get_info(dev)[0]
    widths = [k for k in (1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096) if k * per_col < 0.5 * free_b]
    us_w, best_w = h.tune_batch(widths)
    out["width_sweep"] = {"us_per_iteration": {str(k): round(float(u), 2) for k, u in zip(widths, us_w)},
                          "best_width": widths[best_w],
                          "what": "one iteration (primal + dual step) on N copies of the base LP, plain launches"}

    # B=1 loop: the same kernels, one LP per solve
    b1_n = min(args.b1_lps, q)
    b1_specs = [torch.from_numpy(specs_np[i:i + 1].view(np.uint8).copy()).to(dev) for i in range(b1_n)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b1_solved = 0
    for i in range(b1_n):
        b = h.solve_dev(b1_specs[i], tol=TOL, max_iter=max_iter)
        b1_solved += solved(b.results())
        b.free()
    torch.cuda.synchronize()
    b1_s = time.perf_counter() - t0
    b1_value = b1_solved / b1_s if b1_n > 0 else None
    out["b1_loop"] = {"value": b1_value, "unit": UNIT, "lps": b1_n,
                      "batched_over_b1": value / world / b1_value if b1_value else None}
    h.close()

    # end to end through the public host API: create (H2D of A, vectors),
    # solve from host records, results back to the host
    lp = w.lp
    h2d = (lp.row_ptr.nbytes + lp.col_idx.nbytes + lp.vals.nbytes + lp.c.nbytes + lp.row_lo.nbytes +
           lp.row_hi.nbytes + lp.var_lo.nbytes + lp.var_hi.nbytes + specs_np.nbytes)
    e2e_steps = max(1, min(steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_solved, d2h = 0, 0
    for _ in range(e2e_steps):
        he = lpb.Handle(lp, precision=precision, device=local)
        be = he.solve(specs_np, tol=TOL, max_iter=max_iter)
        r = be.results()
        d2h = r.nbytes
        e2e_solved += solved(r)
        be.free()
        he.close()
    e2e_s = time.perf_counter() - t0
    out["e2e"] = {"value": e2e_solved / e2e_s * world, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                  "d2h_bytes_per_step": int(d2h), "over_value": e2e_solved / e2e_s * world / value,
                  "what": "lpb_create from host CSR + lpb_solve from host records + lpb_results"}
    return out


if __name__ == "__main__":
    main()
