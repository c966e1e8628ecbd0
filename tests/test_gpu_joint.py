"""GPU: the joint solve (lpb_solve_multi), several matrices' batches in one
launch per step (Sec. 5, the batched iteration over LPs of uneven size and
iteration count).

Each batch of a joint solve must come out bitwise as it does alone: the
joint launch gives every row of every matrix to one row group of the width
its batch would launch with alone, summing in the same order, and the
checks, restarts, compaction and polish stay per handle.  The joint results
are also held to the oracle (statuses, objectives within 1e-4 of the
oracle's at rel-KKT 1e-7, and the oracle's KKT of the returned points).
"""
import numpy as np
import pytest

import lpgen

pytestmark = pytest.mark.gpu

GPU_TOL = 1e-5
OBJ_TOL = 1e-4
KKT_TOL = 1e-4
FIELDS = ("status", "restarts", "iters", "obj", "dual_obj", "rel_primal", "rel_dual", "rel_gap", "safe_bound")


@pytest.fixture(scope="module")
def lpb():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2601_21990_gb300 import _build, lpb as mod

    _build.build()
    mod.load()
    return mod


@pytest.fixture(scope="module")
def orc():
    import oracle

    oracle.build()
    return oracle


def _prec(lpb, precision):
    return lpb.FP64 if precision == "fp64" else lpb.MIXED


def uneven_parts():
    """Four matrices of uneven size with batches of uneven width.  FP32 row
    groups: 6 LPs -> 2 lanes, 40 and 50 LPs -> 16 lanes (one launch holds
    both), 136 LPs -> 32 lanes over two column tiles with a ragged second;
    the last matrix has four rows of 2500 entries (ten segments each)."""
    a = lpgen.sb_small(seed=0)
    b = lpgen.sb_powerlaw(seed=3, m=3000, n=7000, children=64)
    c = lpgen.sb_small(seed=1)
    d = lpgen.sb_large(seed=1, m=3000, n=6000, dense_rows=4, dense_len=2500, children=16)
    return [(a.lp, a.specs.subset(np.arange(6))),
            (b.lp, b.specs.subset(np.arange(40))),
            (c.lp, c.specs.subset(np.arange(50) % 16)),
            (d.lp, d.specs.subset(np.arange(136) % 16))]


def assert_same(lpb, alone, joint):
    ra, rj = alone.results(), joint.results()
    for f in FIELDS:
        np.testing.assert_array_equal(ra[f], rj[f], err_msg=f)
    for q in range(alone.num_lps):
        _, xa, ya = alone.result(q)
        _, xj, yj = joint.result(q)
        np.testing.assert_array_equal(xa, xj)
        np.testing.assert_array_equal(ya, yj)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_joint_solve_is_bitwise_the_alone_solve(lpb, precision):
    """Four matrices solved jointly against each solved alone: every result
    field and every x, y bitwise; the joint solve twice (graph replay)."""
    parts = uneven_parts()
    hs = [lpb.Handle(lp, precision=_prec(lpb, precision)) for lp, _ in parts]
    alone = [h.solve(sp, tol=GPU_TOL, max_iter=200000) for h, (_, sp) in zip(hs, parts)]
    for _ in range(2):
        joint = lpb.Handle.solve_multi(hs, [sp for _, sp in parts], tol=GPU_TOL, max_iter=200000)
        for a, j in zip(alone, joint):
            assert_same(lpb, a, j)
    # uneven iteration counts: the batches leave the joint launches at different checks
    its = [int(a.results()["iters"].max()) for a in alone]
    assert len(set(its)) > 1, its


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_joint_solve_against_the_oracle(lpb, orc, precision):
    import os

    parts = uneven_parts()
    hs = [lpb.Handle(lp, precision=_prec(lpb, precision)) for lp, _ in parts]
    joint = lpb.Handle.solve_multi(hs, [sp for _, sp in parts], tol=GPU_TOL, max_iter=200000)
    for (lp, sp), b in zip(parts, joint):
        ref = orc.solve(lp, sp, tol=1e-7, max_iter=400000, threads=os.cpu_count() or 1, lockstep=0)
        res = b.results()
        np.testing.assert_array_equal(res["status"], ref.status)
        opt = np.nonzero(ref.status == 0)[0]
        err = np.abs(res["obj"][opt] - ref.obj[opt]) / (1.0 + np.abs(ref.obj[opt]))
        assert err.size == 0 or err.max() <= OBJ_TOL, (lp.name, err.max())
        for q in opt[:: max(1, len(opt) // 6)]:
            r, x, y = b.result(int(q))
            k = orc.kkt_spec(lp, sp, int(q), x, y, 0)
            assert max(k["rel_primal"], k["rel_dual"], k["rel_gap"]) <= KKT_TOL, (lp.name, q, k)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_joint_solve_with_dense_columns(lpb, precision):
    """A matrix whose columns exceed the long-row threshold (rows of A~^T of
    40 to 1500 entries, over several segments) beside a small one: the joint
    primal launch takes the long-row blocks of A~^T; bitwise as alone."""
    parts = [(lpgen.sb_dense_cols(seed=2), 16), (lpgen.sb_small(seed=6), 40)]
    lps = [(w.lp, w.specs.subset(np.arange(k) % len(w.specs))) for w, k in parts]
    hs = [lpb.Handle(lp, precision=_prec(lpb, precision)) for lp, _ in lps]
    alone = [h.solve(sp, tol=GPU_TOL, max_iter=200000) for h, (_, sp) in zip(hs, lps)]
    joint = lpb.Handle.solve_multi(hs, [sp for _, sp in lps], tol=GPU_TOL, max_iter=200000)
    for a, j in zip(alone, joint):
        assert_same(lpb, a, j)


@pytest.mark.parametrize("graphs,pdl", [(1, 1), (0, 1), (0, 0)])
def test_joint_solve_over_more_than_one_launch_of_parts(lpb, graphs, pdl):
    """Ten matrices of one row-group width: two launches per step (eight
    parts, then two), with and without graphs and programmatic dependent
    launch (the first handle's options); an empty batch among them."""
    ws = [lpgen.sb_small(seed=s) for s in range(10)]
    hs = [lpb.Handle(w.lp, precision=lpb.MIXED, use_graphs=graphs, use_pdl=pdl) for w in ws]
    specs = [w.specs for w in ws]
    specs[4] = ws[4].specs.subset(np.arange(0))
    alone = [h.solve(sp, tol=GPU_TOL, max_iter=200000) for h, sp in zip(hs, specs)]
    joint = lpb.Handle.solve_multi(hs, specs, tol=GPU_TOL, max_iter=200000)
    assert joint[4].num_lps == 0 and joint[4].results().shape[0] == 0
    for a, j in zip(alone, joint):
        assert_same(lpb, a, j)


def test_joint_solve_with_polish(lpb):
    """Batches that stall leave the joint FP32 launches and polish together
    in joint launches on their handles' polish lanes, bitwise as alone.  Two
    handles stall after one check without halving (as the polish test of the
    single solve forces it) and polish in double-float together, a third
    polishes in native FP64, a fourth keeps the defaults."""
    ws = [lpgen.sb_small(seed=3), lpgen.sb_small(seed=4), lpgen.sb_small(seed=5), lpgen.sb_small(seed=2)]
    hs = [lpb.Handle(ws[0].lp, precision=lpb.MIXED, fp64_polish=1, polish_stall_checks=1),
          lpb.Handle(ws[1].lp, precision=lpb.MIXED, fp64_polish=1, polish_stall_checks=1),
          lpb.Handle(ws[2].lp, precision=lpb.MIXED, fp64_polish=1, polish_stall_checks=1,
                     polish_arith=lpb.POLISH_FP64),
          lpb.Handle(ws[3].lp, precision=lpb.MIXED)]
    alone = [h.solve(w.specs, tol=1e-6, max_iter=200000) for h, w in zip(hs, ws)]
    for a in alone[:3]:
        assert a.profile().fp64_switch_iter >= 64
    joint = lpb.Handle.solve_multi(hs, [w.specs for w in ws], tol=1e-6, max_iter=200000)
    for a, j in zip(alone, joint):
        assert a.profile().fp64_switch_iter == j.profile().fp64_switch_iter
        assert_same(lpb, a, j)


def test_joint_polish_near_the_iteration_cap(lpb):
    """The polish phase up to an iteration cap that is not a multiple of the
    check interval (1000 = 15 * 64 + 40): the last joint interval is 40
    iterations long, and each batch stops at the cap as it does alone
    (bitwise), with the LPs still iterating reported at the limit."""
    ws = [lpgen.sb_small(seed=3), lpgen.sb_small(seed=4)]
    hs = [lpb.Handle(ws[0].lp, precision=lpb.MIXED, fp64_polish=1, polish_stall_checks=1),
          lpb.Handle(ws[1].lp, precision=lpb.MIXED, fp64_polish=1, polish_stall_checks=2)]
    cap = 1000
    alone = [h.solve(w.specs, tol=1e-11, max_iter=cap) for h, w in zip(hs, ws)]
    joint = lpb.Handle.solve_multi(hs, [w.specs for w in ws], tol=1e-11, max_iter=cap)
    hit = 0
    for a, j in zip(alone, joint):
        assert_same(lpb, a, j)
        res = j.results()
        assert np.all(res["iters"] <= cap)
        hit += int(np.sum(res["status"] == lpb.ITERATION_LIMIT))
    assert hit > 0


def test_joint_solve_argument_errors(lpb):
    w0, w1 = lpgen.sb_small(seed=0), lpgen.sb_small(seed=1)
    h0 = lpb.Handle(w0.lp, precision=lpb.MIXED)
    h1 = lpb.Handle(w1.lp, precision=lpb.MIXED, check_every=32)
    h2 = lpb.Handle(w1.lp, precision=lpb.FP64)
    for hs in ([h0, h0], [h0, h1], [h0, h2], []):
        with pytest.raises(lpb.LpbError) as e:
            lpb.Handle.solve_multi(hs, [w0.specs] * len(hs))
        assert e.value.code == lpb.LPB_ERR_INVALID_ARG
    bad = w0.specs.subset(np.arange(2))
    bad.kind[1] = 1
    bad.var[1] = w0.lp.n
    with pytest.raises(lpb.LpbError) as e:
        lpb.Handle.solve_multi([h0], [bad])
    assert e.value.code == lpb.LPB_ERR_BAD_INDEX
    # the handles still solve afterwards
    assert h0.solve(w0.specs, tol=1e-4).results()["status"].max() <= 2
