"""Serving (include/lpb_serve.h): continuous batching of requests over
attached matrices.  A request is its own restart group (the batch of Sec. 5),
so its results do not depend on what runs beside it: on matrices whose rows
all take the short-row path the results are bitwise those of lpb_solve on the
same records, alone or in a mix; with long rows (whose block reductions
depend on the batch width) they agree to the solve tolerance."""
import time

import numpy as np
import pytest

import lpgen

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def lpb():
    import torch

    from paper_2601_21990_gb300 import _build, lpb as mod

    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    _build.build()
    mod.load()
    return mod


@pytest.fixture(scope="module")
def orc():
    import oracle

    oracle.build()
    return oracle


def short_row_lp(seed, m=600, n=1200):
    """A strong-branching LP whose rows and columns all have <= 8 nonzeros."""
    rng = np.random.default_rng(seed)
    lengths = rng.integers(3, 9, size=m)
    cols = np.concatenate([rng.choice(n, size=k, replace=False) for k in lengths])
    vals = rng.uniform(0.1, 10.0, size=cols.size) * rng.choice([-1.0, 1.0], size=cols.size)
    row_ptr = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    x0 = rng.uniform(0.0, 10.0, size=n)
    ax = np.zeros(m)
    for i in range(m):
        sl = slice(row_ptr[i], row_ptr[i + 1])
        ax[i] = vals[sl] @ x0[cols[sl]]
    lp = lpgen.LPData(m, n, row_ptr, cols.astype(np.int32), vals, rng.standard_normal(n),
                      ax - rng.uniform(0, 1, size=m), ax + rng.uniform(0, 1, size=m), np.zeros(n),
                      np.full(n, 10.0), x0, "short_rows")
    # every column of A (row of A^T) is short too
    assert np.bincount(lp.col_idx, minlength=n).max() <= 32
    return lp


def child_specs(lp, seed, count):
    rng = np.random.default_rng(seed)
    cand = rng.choice(lp.n, size=(count + 1) // 2, replace=False)
    return lpgen.sb_specs(lp.x0, cand).subset(range(count))


def assert_same_bits(a, b):
    for f in ("status", "iters", "restarts", "obj", "rel_primal", "rel_dual", "rel_gap"):
        np.testing.assert_array_equal(a[f], b[f], err_msg=f)


def test_request_equals_batched_solve_alone_and_in_mix(lpb):
    lp = short_row_lp(1)
    target = child_specs(lp, 7, 24)
    others = [child_specs(lp, 100 + k, c) for k, c in enumerate((40, 7, 64, 19))]
    h_ref = lpb.Handle(lp, precision=lpb.MIXED)
    ref = h_ref.solve(target, tol=TOL, max_iter=64000).results()
    assert np.all(ref["status"] <= 2)

    h = lpb.Handle(lp, precision=lpb.MIXED)
    srv = lpb.Server(lane_columns=256)
    mid = srv.attach(h)
    alone = srv.submit(mid, target, tol=TOL, max_iter=64000)
    srv.wait(alone, 120)
    assert_same_bits(srv.results(alone), ref)

    # the same request among others, admitted while they run
    ids = [srv.submit(mid, others[0], tol=TOL, max_iter=64000), srv.submit(mid, others[1], tol=TOL, max_iter=64000)]
    time.sleep(0.005)
    mixed = srv.submit(mid, target, tol=TOL, max_iter=64000)
    ids += [srv.submit(mid, o, tol=TOL, max_iter=64000) for o in others[2:]]
    for r in ids + [mixed]:
        srv.wait(r, 120)
    assert_same_bits(srv.results(mixed), ref)
    # and each of the others equals its own batched solve
    for sp, r in zip(others, ids):
        assert_same_bits(srv.results(r), h_ref.solve(sp, tol=TOL, max_iter=64000).results())
    st = srv.stats()
    assert st.done == 6 and st.submitted == 6
    srv.close()


def test_power_law_matrix_mix_within_tolerance(lpb, orc):
    """Long rows: alone and in the mix agree to the solve tolerance, and
    every optimal result passes the oracle's KKT evaluation."""
    w = lpgen.sb_powerlaw(seed=2, m=4000, n=8000, children=32)
    h = lpb.Handle(w.lp, precision=lpb.MIXED)
    srv = lpb.Server(lane_columns=128)
    mid = srv.attach(h)
    a = srv.submit(mid, w.specs, tol=TOL, max_iter=100000)
    srv.wait(a, 300)
    ra = srv.results(a)
    rng = np.random.default_rng(5)
    extra = [lpgen.sb_specs(w.lp.x0, rng.choice(w.lp.n, size=k, replace=False)) for k in (20, 8, 30)]
    ids = [srv.submit(mid, extra[0], tol=TOL)]
    b = srv.submit(mid, w.specs, tol=TOL, max_iter=100000)
    ids += [srv.submit(mid, e, tol=TOL) for e in extra[1:]]
    for r in ids + [b]:
        srv.wait(r, 300)
    rb = srv.results(b)
    np.testing.assert_array_equal(ra["status"], rb["status"])
    opt = ra["status"] == 0
    err = np.abs(ra["obj"][opt] - rb["obj"][opt]) / (1.0 + np.abs(ra["obj"][opt]))
    assert err.max() <= TOL, err.max()
    for q in np.nonzero(rb["status"] == 0)[0][:6]:
        r, x, y = srv.result(b, mid, int(q))
        k = orc.kkt_spec(w.lp, w.specs, int(q), x, y)
        assert max(k["rel_primal"], k["rel_dual"], k["rel_gap"]) <= TOL, (q, k)
    srv.close()


def test_continuous_admission_and_two_matrices(lpb):
    """Requests arriving while others run are admitted between intervals;
    two matrices run side by side; each result equals its batched solve."""
    lp1, lp2 = short_row_lp(3), short_row_lp(4, m=900, n=1500)
    h1, h2 = lpb.Handle(lp1, precision=lpb.MIXED), lpb.Handle(lp2, precision=lpb.MIXED)
    srv = lpb.Server(lane_columns=128)
    m1, m2 = srv.attach(h1), srv.attach(h2)
    reqs = []
    for k in range(10):
        lp, mid = (lp1, m1) if k % 2 == 0 else (lp2, m2)
        sp = child_specs(lp, 200 + k, 5 + 7 * k)
        reqs.append((mid, lp, sp, srv.submit(mid, sp, tol=TOL, max_iter=64000)))
        time.sleep(0.002)
    for mid, lp, sp, r in reqs:
        srv.wait(r, 120)
        info = srv.info(r)
        assert info.state == lpb.REQ_DONE and info.t_submit <= info.t_admit <= info.t_done
        ref = lpb.Handle(lp, precision=lpb.MIXED).solve(sp, tol=TOL, max_iter=64000).results()
        assert_same_bits(srv.results(r), ref)
    st = srv.stats()
    assert st.admitted_while_busy >= 1, (st.admitted_while_busy, st.intervals)
    srv.close()


def test_warm_start_from_parent_on_device(lpb, orc):
    """Children start from the parent's solution kept on the device."""
    w = lpgen.sb_small(seed=0)
    h = lpb.Handle(w.lp, precision=lpb.MIXED)
    srv = lpb.Server(lane_columns=64)
    mid = srv.attach(h)
    parent = srv.submit(mid, lpb.specs_array([0], [-1]), tol=1e-6, max_iter=200000)
    children = srv.submit(mid, w.specs, tol=TOL, max_iter=200000, warm_request=parent, warm_lp=0)
    cold = srv.submit(mid, w.specs, tol=TOL, max_iter=200000)
    for r in (parent, children, cold):
        srv.wait(r, 120)
    rw, rc = srv.results(children), srv.results(cold)
    np.testing.assert_array_equal(rw["status"], rc["status"])
    opt = rc["status"] == 0
    assert np.all(np.abs(rw["obj"][opt] - rc["obj"][opt]) <= 1e-3 * (1 + np.abs(rc["obj"][opt])))
    for q in np.nonzero(rw["status"] == 0)[0]:
        r, x, y = srv.result(children, mid, int(q))
        k = orc.kkt_spec(w.lp, w.specs, int(q), x, y)
        assert max(k["rel_primal"], k["rel_dual"], k["rel_gap"]) <= TOL, (q, k)
    # the warm start must not be released while a request waits on it
    srv.release(children)
    srv.release(parent)
    with pytest.raises(lpb.LpbError):
        srv.submit(mid, w.specs, tol=TOL, warm_request=parent, warm_lp=0)
    srv.close()


def test_budget_limits_admission(lpb):
    """With an HBM budget that holds one request's buffers at a time, the
    others wait in the queue and all finish."""
    lp = short_row_lp(6)
    h = lpb.Handle(lp, precision=lpb.MIXED)
    lane = 128 * (5 * lp.n + 5 * lp.m) * 4 + 128 * 256 + 64 * (5 * lp.n + 5 * lp.m) * 8 + 64 * 256
    per_req = 24 * (lp.n + lp.m) * 8 + 24 * 32
    srv = lpb.Server(lane_columns=128, polish_columns=64, hbm_budget_bytes=lane + per_req + per_req // 2)
    mid = srv.attach(h)
    ids = [srv.submit(mid, child_specs(lp, 300 + k, 24), tol=TOL, max_iter=64000) for k in range(4)]
    for k, r in enumerate(ids):
        srv.wait(r, 120)
        srv.release(r)
    infos = [srv.info(r) for r in ids]
    # admitted one after another: each starts after the previous finished
    for a, b in zip(infos, infos[1:]):
        assert b.t_admit >= a.t_done - 1e-6
    srv.close()


def test_stalled_request_moves_to_polish_lane(lpb, orc):
    """At tol 1e-7 the FP32 iterates stall; the request moves to the
    double-float polish lane and finishes there."""
    w = lpgen.sb_small(seed=3)
    h = lpb.Handle(w.lp, precision=lpb.MIXED, polish_stall_checks=4)
    srv = lpb.Server(lane_columns=64, polish_columns=32)
    mid = srv.attach(h)
    r = srv.submit(mid, w.specs, tol=1e-7, max_iter=400000)
    srv.wait(r, 300)
    info = srv.info(r)
    assert info.polished == 1 and srv.stats().migrations >= 1
    res = srv.results(r)
    for q in np.nonzero(res["status"] == 0)[0][:8]:
        rr, x, y = srv.result(r, mid, int(q))
        k = orc.kkt_spec(w.lp, w.specs, int(q), x, y)
        assert max(k["rel_primal"], k["rel_dual"], k["rel_gap"]) <= 1e-6, (q, k)
    srv.close()


def test_bad_requests_are_rejected(lpb):
    lp = short_row_lp(8)
    h = lpb.Handle(lp, precision=lpb.MIXED)
    srv = lpb.Server(lane_columns=32)
    mid = srv.attach(h)
    with pytest.raises(lpb.LpbError):
        srv.submit(mid, lpb.specs_array([1], [lp.n + 5], [0.0], [1.0]))
    with pytest.raises(lpb.LpbError):
        srv.submit(mid + 3, lpb.specs_array([0], [-1]))
    with pytest.raises(lpb.LpbError):
        srv.submit(mid, lpb.specs_array([0] * 40, [-1] * 40))  # more LPs than lane columns
    r = srv.submit(mid, lpb.specs_array([0], [-1]), tol=TOL)
    srv.wait(r, 60)
    assert srv.results(r)["status"][0] == 0
    srv.close()


def test_polish_moves_beside_running_requests(lpb, orc):
    """A request that stalls moves to the polish lane while other requests
    keep running (and finish, and compact) in the FP32 lane of the same
    matrix: every request finishes with results the oracle accepts."""
    w = lpgen.sb_small(seed=3)
    h = lpb.Handle(w.lp, precision=lpb.MIXED, polish_stall_checks=4)
    srv = lpb.Server(lane_columns=96, polish_columns=32)
    mid = srv.attach(h)
    rng = np.random.default_rng(11)
    tight = srv.submit(mid, w.specs, tol=1e-7, max_iter=400000)
    loose = [srv.submit(mid, lpgen.sb_specs(w.lp.x0, rng.choice(w.lp.n, size=k, replace=False)), tol=TOL,
                        max_iter=400000) for k in (6, 9, 12, 7)]
    for r in [tight] + loose:
        srv.wait(r, 300)
    assert srv.info(tight).polished == 1
    for r, tol in [(tight, 1e-6)] + [(q, TOL) for q in loose]:
        res = srv.results(r)
        sp = w.specs if r == tight else None
        assert np.all(res["status"] <= 3)
        if sp is not None:
            for q in np.nonzero(res["status"] == 0)[0][:6]:
                rr, x, y = srv.result(r, mid, int(q))
                k = orc.kkt_spec(w.lp, sp, int(q), x, y)
                assert max(k["rel_primal"], k["rel_dual"], k["rel_gap"]) <= tol, (q, k)
    assert srv.stats().migrations >= 1
    srv.close()
