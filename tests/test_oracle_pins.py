"""Pins for the FP64 CPU oracle against things the paper and mathematics fix.

Each test pins the oracle to something other than itself: hand-computed
vectors, published generator outputs, closed-form LPs, brute-force vertex
enumeration, an independent LP solver (HiGHS via scipy), LP duality and the
firm nonexpansiveness of the PDHG operator.  ``test_planted_mistakes_are_caught``
plants known mistakes in the oracle and checks that some pin fails for each.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import handcases
import lpgen

INF = np.inf
HERE = os.path.dirname(os.path.abspath(__file__))


def _f(v):
    return float(v) if not isinstance(v, str) else float(v.replace("inf", "inf"))


# ---------------------------------------------------------------------------
# Sec. 3 primitives: hand-computed vectors
# ---------------------------------------------------------------------------

def test_projection_hand_vectors(oracle_lib):
    o = oracle_lib
    v = [-3.0, 0.5, 7.0, -2.0, 4.0, -1.0, 2.0]
    a = [-1.0, 0.0, 1.0, -INF, -INF, 0.0, -INF]
    b = [1.0, 1.0, 5.0, 3.0, INF, INF, INF]
    np.testing.assert_array_equal(o.project_box(v, a, b), [-1.0, 0.5, 5.0, -2.0, 4.0, 0.0, 2.0])
    # barrier cone: v >= 0 where a=-inf, v <= 0 where b=+inf, {0} where both infinite
    np.testing.assert_array_equal(o.project_barrier(v, a, b), [-3.0, 0.5, 7.0, 0.0, 0.0, -1.0, 0.0])
    # recession cone: {0} for finite intervals, R_- for (-inf,b], R_+ for [a,inf), R for R
    np.testing.assert_array_equal(o.project_recession(v, a, b), [0.0, 0.0, 0.0, -2.0, 4.0, 0.0, 2.0])


def test_support_function_hand_values(oracle_lib):
    o = oracle_lib
    # phi_[a,b](v) = b^T v_+ + a^T v_-, with 0 * inf = 0
    assert o.support([2.0, -3.0, 0.0, 1.5], [-1.0, 2.0, -INF, -INF], [4.0, 5.0, 7.0, 3.0]) == 6.5
    assert o.support([0.0, 0.0], [-INF, -INF], [INF, INF]) == 0.0
    assert o.support([-1.0], [-INF], [3.0]) == INF  # v outside the barrier cone
    assert o.support([1.0], [0.0], [INF]) == INF


def test_robust_reduced_cost_hand_vectors(oracle_lib):
    # v > 0 pairs with the upper bound b, v < 0 with the lower bound a; kept
    # only where that bound is finite and |x - bound| <= |x|
    v = [1.0, 1.0, -1.0, -1.0, 0.0, 2.0, 3.0, -2.0, 1.0]
    x = [0.0, 9.0, 0.0, 3.0, 5.0, 5.0, -4.0, -4.0, 2.0]
    a = [0.0, 0.0, 0.0, -1e300, 0.0, 0.0, -5.0, -5.0, -INF]
    b = [1e10, 10.0, 1e10, 10.0, 10.0, 10.0, -3.0, -3.0, INF]
    np.testing.assert_array_equal(oracle_lib.robust_reduced_cost(v, x, a, b),
                                  [0.0, 1.0, -1.0, 0.0, 0.0, 2.0, 3.0, -2.0, 0.0])
    # with x on the bound v pairs with, it is Pi_B(v)
    va = np.array([0.7, -0.3, 1.5, -2.5])
    lo = np.array([-2.0, -2.0, 1.0, 1.0])
    hi = np.array([3.0, 3.0, 4.0, 4.0])
    xs = np.where(va > 0, hi, lo)
    np.testing.assert_array_equal(oracle_lib.robust_reduced_cost(va, xs, lo, hi),
                                  oracle_lib.project_barrier(va, lo, hi))


def test_splitmix64_published_outputs(oracle_lib):
    # SplitMix64 seeded with 0 (Steele, Lea, Flood 2014; reference code by Vigna)
    assert oracle_lib.splitmix64_at(0, 0) == 0xE220A8397B1DCDAF
    assert oracle_lib.splitmix64_at(0, 1) == 0x6E789E6AA1B965F4
    assert oracle_lib.splitmix64_at(0, 2) == 0x06C45D188009454F


def test_kkt_handworked_golden(oracle_lib):
    g = json.load(open(os.path.join(HERE, "golden", "kkt_handworked.json")))
    lpd = g["lp"]
    for case in g["cases"]:
        lp = lpgen.from_dense(lpd["A"], lpd["c"], [_f(v) for v in lpd["row_lo"]],
                              [_f(v) for v in lpd["row_hi"]], [_f(v) for v in case["var_lo"]],
                              [_f(v) for v in case["var_hi"]])
        k = oracle_lib.kkt(lp, 0, 0, 0.0, 0.0, 1.0, case["x"], case["y"])
        for key in ("obj", "dual_obj", "rel_primal", "rel_dual", "rel_gap"):
            want = _f(case[key])
            if math.isinf(want):
                assert k[key] == want, (case["name"], key)
            else:
                assert k[key] == pytest.approx(want, abs=1e-14, rel=1e-12), (case["name"], key)


def _robust_cases():
    g = json.load(open(os.path.join(HERE, "golden", "kkt_robust_handworked.json")))
    lpd = g["lp"]
    for case in g["cases"]:
        lp = lpgen.from_dense(lpd["A"], lpd["c"], [_f(v) for v in lpd["row_lo"]],
                              [_f(v) for v in lpd["row_hi"]], [_f(v) for v in case["var_lo"]],
                              [_f(v) for v in case["var_hi"]])
        yield case, lp


def test_kkt_robust_reduced_cost_handworked_golden(oracle_lib):
    for case, lp in _robust_cases():
        for mode, want in case["modes"].items():
            k = oracle_lib.kkt(lp, 0, 0, 0.0, 0.0, 1.0, case["x"], case["y"], reduced_cost=int(mode))
            for key, v in want.items():
                assert k[key] == pytest.approx(_f(v), abs=1e-14, rel=1e-12), (case["name"], mode, key)


def test_robust_reduced_cost_knapsack_with_huge_bounds(oracle_lib):
    """Upper bounds of 1e10 that no optimum reaches: the robust stopping test
    meets a tight tolerance at the greedy closed form."""
    rng = np.random.default_rng(5)
    n = 8
    a = rng.uniform(0.5, 3, n)
    c = rng.uniform(0.5, 3, n)
    b = 4.0
    i = int(np.argmin(c / a))
    f = c[i] * b / a[i]  # all coverage from the cheapest variable per unit
    lp = lpgen.from_dense(a[None, :], c, [b], [INF], np.zeros(n), np.full(n, 1e10))
    r = oracle_lib.solve(lp, lpgen.base_specs(1), tol=1e-8, max_iter=200000, check_every=16, reduced_cost=1)
    assert r.status[0] == 0
    assert r.obj[0] == pytest.approx(f, rel=1e-6)
    k = oracle_lib.kkt(lp, 0, 0, 0.0, 0.0, 1.0, r.x[0], r.y[0], reduced_cost=1)
    assert max(k["rel_primal"], k["rel_dual"], k["rel_gap"]) <= 1e-8


def test_robust_reduced_cost_large_bounds_against_highs(oracle_lib):
    """Covering LPs whose 1e10 upper bounds no optimum reaches: with the
    robust reduced cost every child meets 1e-7 at HiGHS's objective; with
    Pi_B as printed, the bounds' share of the dual objective keeps the gap
    open under the same iteration cap."""
    w = lpgen.covering_large_bounds(seed=0)
    r = oracle_lib.solve(w.lp, w.specs, tol=1e-7, max_iter=50000, lockstep=0, threads=4, reduced_cost=1)
    assert np.all(r.status == 0)
    for q in range(len(w.specs)):
        st, f = highs_solve(w.lp, w.specs, q)
        assert st == 0 and abs(r.obj[q] - f) / (1 + abs(f)) <= 1e-6, (q, r.obj[q], f)
    r0 = oracle_lib.solve(w.lp, w.specs.subset(range(4)), tol=1e-7, max_iter=50000, lockstep=0, threads=4)
    assert np.all(r0.status == 3)
    assert np.all(r0.rel_gap > 1e-6)


# ---------------------------------------------------------------------------
# ||A||_2 and scaling
# ---------------------------------------------------------------------------

def test_norm_estimate_matches_svd(oracle_lib):
    for seed in range(4):
        lp = lpgen.random_lp(seed, 12 + seed, 9 + 2 * seed, density=0.4)
        est, it = oracle_lib.norm2_estimate(lp)
        exact = np.linalg.norm(lp.dense(), 2)
        assert est == pytest.approx(exact, rel=1e-7), (seed, it)
        assert est <= exact * (1 + 1e-12)  # Rayleigh quotient never overshoots


def test_ruiz_diagonal_closed_form(oracle_lib):
    d = np.array([4.0, 0.25, 9.0])
    lp = lpgen.from_dense(np.diag(d), np.ones(3), -np.ones(3), np.ones(3), -np.ones(3), np.ones(3))
    dr, dc = oracle_lib.scaling(lp, ruiz_iters=1, pock_chambolle=False)
    np.testing.assert_allclose(dr, 1 / np.sqrt(d), rtol=1e-15)
    np.testing.assert_allclose(dc, 1 / np.sqrt(d), rtol=1e-15)
    # Pock-Chambolle on the identity leaves it unchanged
    dr2, dc2 = oracle_lib.scaling(lp, ruiz_iters=1, pock_chambolle=True)
    np.testing.assert_allclose(dr2 * d * dc2, np.ones(3), rtol=1e-15)


def test_pock_chambolle_pass_by_hand(oracle_lib):
    """Reading R1: one Pock-Chambolle pass (alpha = 1) divides each row and
    column by the square root of its absolute sum, both sums taken from the
    same matrix; alone and after one Ruiz pass, on a 2 x 2 matrix with the
    factors written out by hand (tests/handcases.py)."""
    for a, ruiz, dr_want, dc_want in handcases.pc_cases():
        lp = lpgen.from_dense(a, [1.0, 1.0], [-1.0, -1.0], [1.0, 1.0], [0.0, 0.0], [1.0, 1.0])
        dr, dc = oracle_lib.scaling(lp, ruiz_iters=ruiz, pock_chambolle=True)
        np.testing.assert_allclose(dr, dr_want, rtol=1e-14)
        np.testing.assert_allclose(dc, dc_want, rtol=1e-14)


def test_ruiz_fixed_point_unit_inf_norms(oracle_lib):
    lp = lpgen.random_lp(3, 15, 11, density=0.5)
    dr, dc = oracle_lib.scaling(lp, ruiz_iters=60, pock_chambolle=False)
    a = np.abs(dr[:, None] * lp.dense() * dc[None, :])
    np.testing.assert_allclose(a.max(axis=1), 1.0, atol=1e-6)
    np.testing.assert_allclose(a.max(axis=0), 1.0, atol=1e-6)


def test_zero_rows_and_columns_keep_unit_scale(oracle_lib):
    a = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 8.0]])
    lp = lpgen.from_dense(a, [1, 1, 1], [-1, -1], [1, 1], [0, 0, 0], [1, 1, 1])
    dr, dc = oracle_lib.scaling(lp)
    assert dr[0] == 1.0 and dc[1] == 1.0


# ---------------------------------------------------------------------------
# PDHG operator: firm nonexpansiveness in the M-norm (reading R4, minus sign)
# ---------------------------------------------------------------------------

def _t_data(seed):
    lp = lpgen.random_lp(seed, 7, 9, density=0.5)
    est = np.linalg.norm(lp.dense(), 2)
    return lp, 0.998 / est


def test_T_is_nonexpansive_in_M_norm(oracle_lib):
    o = oracle_lib
    rng = np.random.default_rng(0)
    for seed in range(5):
        lp, eta = _t_data(seed)
        for w in (0.3, 1.0, 4.0):
            tau, sigma = eta / w, eta * w
            for _ in range(40):
                z1 = rng.normal(size=lp.n) * 3, rng.normal(size=lp.m) * 3
                z2 = rng.normal(size=lp.n) * 3, rng.normal(size=lp.m) * 3
                t1 = o.apply_T(lp, lp.c, lp.var_lo, lp.var_hi, lp.row_lo, lp.row_hi, tau, sigma, *z1)
                t2 = o.apply_T(lp, lp.c, lp.var_lo, lp.var_hi, lp.row_lo, lp.row_hi, tau, sigma, *z2)
                before = o.mnorm2(lp, w, eta, -1.0, z1[0] - z2[0], z1[1] - z2[1])
                after = o.mnorm2(lp, w, eta, -1.0, t1[0] - t2[0], t1[1] - t2[1])
                assert before > 0
                assert after <= before * (1 + 1e-12) + 1e-12


def _translation_lp():
    """One variable, no rows, box [-1, 1], cost 1e-3: with no rows ||A~|| = 0,
    so eta = 0.998 and w = 1 (readings R2, R3), tau = 0.998, and the PDHG
    operator is the translation T(z) = z - delta, delta = tau * 1e-3, until
    the box is reached."""
    return lpgen.from_dense(np.zeros((0, 1)), [1e-3], [], [], [-1.0], [1.0])


def test_halpern_trajectory_closed_form(oracle_lib):
    """Eq. mainiter on a translation, solved in closed form: with
    z^{k+1} = (k+1)/(k+2) (2 T(z^k) - z^k) + z^0/(k+2) and T(z) = z - delta,
    (k+2) z^{k+1} = (k+1) (z^k - 2 delta) + z^0 gives z^k = z^0 - k delta, so
    the point evaluated at the K-th check, T(z^{K-1}), is z^0 - K delta.
    Restarts are switched off (beta_s = beta_n = 0, beta_a = 1e9) and every
    iteration is a check, so the solve stops at the iteration limit K."""
    lp = _translation_lp()
    delta = 0.998e-3
    for K in (1, 2, 3, 7, 50, 400):
        r = oracle_lib.solve(lp, lpgen.base_specs(1), tol=1e-12, max_iter=K, check_every=1,
                             detect_infeasibility=0, beta_s=0.0, beta_n=0.0, beta_a=1e9,
                             warm_x=[0.5], warm_y=np.zeros(0))
        assert r.status[0] == 3 and r.iters[0] == K and r.restarts[0] == 0
        assert r.x[0][0] == pytest.approx(0.5 - K * delta, abs=1e-14)
    # the dual side: x fixed at 0, one row x >= 1 (infeasible; detection off),
    # c = 0 so w = 1 and sigma = eta = 0.998; the dual operator is the
    # translation y -> y - sigma, so the K-th evaluated y is y^0 - K sigma
    lp = lpgen.from_dense(np.ones((1, 1)), [0.0], [1.0], [np.inf], [0.0], [0.0])
    for K in (1, 2, 7, 50):
        r = oracle_lib.solve(lp, lpgen.base_specs(1), tol=1e-12, max_iter=K, check_every=1,
                             detect_infeasibility=0, beta_s=0.0, beta_n=0.0, beta_a=1e9,
                             warm_x=[0.0], warm_y=[-0.25])
        assert r.status[0] == 3 and r.iters[0] == K and r.restarts[0] == 0
        assert r.x[0][0] == 0.0
        assert r.y[0][0] == pytest.approx(-0.25 - K * 0.998, abs=1e-12)


def test_restart_schedule_by_hand(oracle_lib):
    """Sec. 4 "Restarts" in reading R5, on the translation LP, whose fixed-point
    residual is the same at every check, so conditions (i) and (ii) fire only
    when their beta is 1.  Checks every 4 iterations, 72 iterations; a check
    at global index K (0-based) with inner index k restarts when k > beta_a K,
    then k = 0, else k + 1; the last check ends the solve without a restart.
    - beta_a = 0.36, beta_s = beta_n = 0: the checks at K = 3, 7, 11, ... see
      k = 3 (> 1.08, restart), 3 (> 2.52, restart), 3 (< 3.96), 7 (> 5.4,
      restart), 3, 7, 11 (> 9.72, restart), 3, 7, 11, 15, 19 (> 16.92,
      restart), 3, 7, 11, 15, 19, 23 (K = 71, last): 5 restarts.
    - beta_s = 1: every check but the last restarts: 18 checks, 17 restarts.
    Restarting a translation at T(z) continues the same line, so the point is
    still z^0 - K delta."""
    lp = _translation_lp()
    for kw, want in ((dict(beta_s=0.0, beta_n=0.0, beta_a=0.36), 5), (dict(beta_s=1.0, beta_n=0.0, beta_a=1e9), 17)):
        r = oracle_lib.solve(lp, lpgen.base_specs(1), tol=1e-12, max_iter=72, check_every=4, detect_infeasibility=0,
                             warm_x=[0.5], warm_y=np.zeros(0), **kw)
        assert r.status[0] == 3 and r.iters[0] == 72
        assert r.restarts[0] == want, kw
        assert r.x[0][0] == pytest.approx(0.5 - 72 * 0.998e-3, abs=1e-14)


def _restart_batch_solve(o, beta_n, mutation=0):
    lp, specs, wx, wy = handcases.restart_batch()
    return o.solve(lp, specs, tol=1e-12, max_iter=handcases.RESTART_BATCH_MAX_ITER, lockstep=1, warm_x=wx,
                   warm_y=wy, beta_n=beta_n, mutation=mutation, **handcases.RESTART_BATCH_KW)


def test_restart_conditions_and_active_mean_by_hand(oracle_lib):
    """Sec. 4 "Restarts" condition (ii) and Sec. 5's batch-averaged residual
    over the LPs still active (reading R11), on the five-LP lockstep batch of
    tests/handcases.py: the mean residual falls at check 2 and rises at
    check 3 while below beta_n r0, so condition (ii) restarts at check 3 for
    beta_n = 0.9 and nothing restarts for beta_n = 0.5.  The statuses,
    finishing iterations and optimal points are derived by hand as well."""
    for beta_n, want in handcases.RESTART_BATCH_RESTARTS.items():
        r = _restart_batch_solve(oracle_lib, beta_n)
        assert r.status.tolist() == handcases.RESTART_BATCH_STATUS
        assert r.iters.tolist() == handcases.RESTART_BATCH_ITERS
        assert r.restarts.tolist() == want, beta_n
        for q, xq in handcases.RESTART_BATCH_OPT_X.items():
            np.testing.assert_allclose(r.x[q], xq, atol=1e-15)


def test_primal_weight_update_by_hand(oracle_lib):
    """Sec. 4 "Step-size and primal weight" in readings R3 and R6/R7, by hand.
    x1 moves freely with cost 0.3; x2 is fixed at 0 under the row x2 >= 2
    (infeasible, detection off); x3 is fixed at 0 with cost 0.4.  A = [0 1 0]
    needs no scaling and ||A|| = 1, so eta = 0.998; w0 = ||c|| / ||b|| =
    0.5 / 2.  From z0 = 0 the first step gives dx = -tau0 c1 (x1 only) and
    dy = -2 sigma0 (y^ = sigma (v - Pi(v)) with v = 0, Pi(v) = 2).  beta_s = 1
    restarts at that first check: d = ||dy|| / ||dx|| = 2 w0^2 / c1 and
    w1 = exp(theta log d + (1 - theta) log w0) with theta = 1/2.  The second
    and last iteration steps from the new anchor with tau1 = eta / w1,
    sigma1 = eta w1, so x1 = -c1 (tau0 + tau1) and y = -2 (sigma0 + sigma1).
    The printed ratio ||dx|| / ||dy|| would give x1 = -1.584 instead of -2.125."""
    lp = lpgen.from_dense(np.array([[0.0, 1.0, 0.0]]), [0.3, 0.0, 0.4], [2.0], [INF], [-1e6, 0.0, 0.0],
                          [1e6, 0.0, 0.0])
    eta, c1, w0 = 0.998, 0.3, 0.25
    d = 2 * w0 ** 2 / c1
    w1 = math.exp(0.5 * math.log(d) + 0.5 * math.log(w0))
    r = oracle_lib.solve(lp, lpgen.base_specs(1), tol=1e-12, max_iter=2, check_every=1, detect_infeasibility=0,
                         beta_s=1.0, beta_n=0.0, beta_a=1e9, warm_x=[0.0, 0.0, 0.0], warm_y=[0.0])
    assert r.eta == pytest.approx(eta, rel=1e-12)
    assert r.status[0] == 3 and r.iters[0] == 2 and r.restarts[0] == 1
    assert r.x[0][0] == pytest.approx(-c1 * (eta / w0 + eta / w1), rel=1e-12)
    assert r.y[0][0] == pytest.approx(-2 * (eta * w0 + eta * w1), rel=1e-12)


def test_fixed_point_residual_zero_at_optimum(oracle_lib):
    """At a primal-dual optimum z*, T(z*) = z* (hand LP of the KKT golden)."""
    o = oracle_lib
    lp = lpgen.from_dense([[1.0, 2.0]], [1.0, 1.0], [2.0], [INF], [0, 0], [10, 10])
    x, y = np.array([0.0, 1.0]), np.array([-0.5])
    for tau, sigma in ((0.1, 0.3), (0.4, 0.2)):
        xh, yh = o.apply_T(lp, lp.c, lp.var_lo, lp.var_hi, lp.row_lo, lp.row_hi, tau, sigma, x, y)
        np.testing.assert_allclose(xh, x, atol=1e-15)
        np.testing.assert_allclose(yh, y, atol=1e-15)


# ---------------------------------------------------------------------------
# whole-solver pins
# ---------------------------------------------------------------------------

def highs_solve(lp, specs, q):
    from scipy.optimize import linprog
    a = lp.dense()
    xl, xu, c = lp.var_lo.copy(), lp.var_hi.copy(), lp.c.copy()
    j = int(specs.var[q])
    if specs.kind[q] == lpgen.KIND_BOUND:
        xl[j] = max(xl[j], specs.lo[q])
        xu[j] = min(xu[j], specs.hi[q])
    elif specs.kind[q] == lpgen.KIND_OBJECTIVE:
        c = np.zeros(lp.n)
        c[j] = specs.sign[q]
    fu, fl = np.isfinite(lp.row_hi), np.isfinite(lp.row_lo)
    aub = np.vstack([a[fu], -a[fl]]) if lp.m else None
    bub = np.concatenate([lp.row_hi[fu], -lp.row_lo[fl]]) if lp.m else None
    if bub is not None and bub.size == 0:
        aub = bub = None
    bounds = [(None if np.isinf(l) else l, None if np.isinf(u) else u) for l, u in zip(xl, xu)]
    r = linprog(c, A_ub=aub, b_ub=bub, bounds=bounds, method="highs")
    return r.status, (r.fun if r.status == 0 else None)


def test_box_lp_closed_form(oracle_lib):
    rng = np.random.default_rng(1)
    n = 9
    lo = rng.uniform(-5, 0, n)
    hi = lo + rng.uniform(0.5, 4, n)
    c = rng.normal(size=n)
    lp = lpgen.from_dense(np.zeros((0, n)), c, [], [], lo, hi)
    r = oracle_lib.solve(lp, lpgen.base_specs(1), tol=1e-10, max_iter=10000, check_every=8)
    assert r.status[0] == 0
    np.testing.assert_allclose(r.x[0], np.where(c > 0, lo, hi), atol=1e-9)
    assert r.obj[0] == pytest.approx(np.minimum(c * lo, c * hi).sum(), abs=1e-9)
    # OBBT on a box returns the box
    cand = np.arange(n)
    ro = oracle_lib.solve(lp, lpgen.obbt_specs(cand), tol=1e-10, max_iter=10000, check_every=8)
    np.testing.assert_allclose(ro.obj[:n], lo, atol=1e-8)
    np.testing.assert_allclose(-ro.obj[n:], hi, atol=1e-8)


def test_continuous_knapsack_closed_form(oracle_lib):
    rng = np.random.default_rng(2)
    n = 8
    a = rng.uniform(0.5, 3, n)
    c = rng.uniform(0.5, 3, n)
    u = rng.uniform(0.5, 2, n)
    b = 0.55 * (a * u).sum()
    # greedy: cheapest cost per unit of coverage first
    f, need = 0.0, b
    for i in np.argsort(c / a):
        take = min(u[i], need / a[i])
        f += c[i] * take
        need -= a[i] * take
        if need <= 0:
            break
    lp = lpgen.from_dense(a[None, :], c, [b], [INF], np.zeros(n), u)
    r = oracle_lib.solve(lp, lpgen.base_specs(1), tol=1e-9, max_iter=200000, check_every=16)
    assert r.status[0] == 0
    assert r.obj[0] == pytest.approx(f, rel=1e-7)


def brute_force_vertices(a, c, l, u, xl, xu):
    """min c^T x over the polytope, by enumerating all vertices: choose n
    active hyperplanes among {row at l or u, variable at its lower or upper
    bound}, solve, keep the feasible points.  Returns None when no vertex is
    feasible (the box is bounded, so the LP is then infeasible)."""
    m, n = a.shape
    planes = []
    for i in range(m):
        planes.append((a[i], l[i]))
        planes.append((a[i], u[i]))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        planes.append((e, xl[j]))
        planes.append((e, xu[j]))
    best = None
    for comb in itertools.combinations(range(len(planes)), n):
        mat = np.array([planes[k][0] for k in comb])
        if abs(np.linalg.det(mat)) < 1e-10:
            continue
        x = np.linalg.solve(mat, np.array([planes[k][1] for k in comb]))
        ax = a @ x
        if np.all(ax >= l - 1e-9) and np.all(ax <= u + 1e-9) and np.all(x >= xl - 1e-9) and np.all(x <= xu + 1e-9):
            f = c @ x
            best = f if best is None else min(best, f)
    return best


@pytest.mark.parametrize("seed", range(8))
def test_brute_force_vertex_enumeration(oracle_lib, seed):
    rng = np.random.default_rng(100 + seed)
    m, n = 2 + seed % 3, 3 + seed % 3
    a = np.round(rng.uniform(-3, 3, (m, n)), 1)
    x0 = rng.uniform(0, 1, n)
    xl, xu = np.zeros(n), np.ones(n)
    l = a @ x0 - rng.uniform(0, 0.3, m)
    u = a @ x0 + rng.uniform(0, 0.3, m)
    if seed % 4 == 3:  # make it infeasible: a row range out of reach
        l[0] = u[0] = np.abs(a[0]).sum() + 1.0
    c = rng.normal(size=n)
    f = brute_force_vertices(a, c, l, u, xl, xu)
    lp = lpgen.from_dense(a, c, l, u, xl, xu)
    r = oracle_lib.solve(lp, lpgen.base_specs(1), tol=1e-9, max_iter=400000, check_every=16)
    if f is None:
        assert r.status[0] == 1  # PRIMAL_INFEASIBLE
    else:
        assert r.status[0] == 0
        assert r.obj[0] == pytest.approx(f, abs=1e-6 * (1 + abs(f)))


def test_sb_small_against_highs(oracle_lib):
    w = lpgen.sb_small()
    r = oracle_lib.solve(w.lp, w.specs, tol=1e-8, max_iter=200000)
    for q in range(len(w.specs)):
        st, f = highs_solve(w.lp, w.specs, q)
        assert st == 0 and r.status[q] == 0
        assert abs(r.obj[q] - f) / (1 + abs(f)) <= 1e-7, q


@pytest.mark.parametrize("seed", range(12))
def test_mixed_bound_lps_against_highs(oracle_lib, seed):
    lp = lpgen.random_lp(seed, 4 + seed % 5, 6 + seed % 4)
    sp = lpgen.base_specs(1)
    r = oracle_lib.solve(lp, sp, tol=1e-8, max_iter=400000, check_every=16)
    st, f = highs_solve(lp, sp, 0)
    assert r.status[0] == {0: 0, 2: 1, 3: 2}[st]  # HiGHS optimal / infeasible / unbounded
    if st == 0:
        assert abs(r.obj[0] - f) / (1 + abs(f)) <= 1e-6


@pytest.mark.parametrize("seed", range(8))
def test_robust_reduced_cost_mixed_bounds_against_highs(oracle_lib, seed):
    """Robust-mode stopping on every bound type (free, one-sided and fixed
    variables; equality, ranged and one-sided rows) reaches HiGHS's optimum
    and the same status; with the far side of some boxes moved out to 1e9 the
    optimum is unchanged when HiGHS says so."""
    lp = lpgen.random_lp(seed, 4 + seed % 5, 6 + seed % 4)
    sp = lpgen.base_specs(1)
    st, f = highs_solve(lp, sp, 0)
    r = oracle_lib.solve(lp, sp, tol=1e-8, max_iter=400000, check_every=16, reduced_cost=1)
    assert r.status[0] == {0: 0, 2: 1, 3: 2}[st]
    if st != 0:
        return
    assert abs(r.obj[0] - f) / (1 + abs(f)) <= 1e-6
    k = oracle_lib.kkt(lp, 0, 0, 0.0, 0.0, 1.0, r.x[0], r.y[0], reduced_cost=1)
    assert max(k["rel_primal"], k["rel_dual"], k["rel_gap"]) <= 1e-8
    # widen the inactive side of each two-sided box to 1e9
    x = r.x[0]
    lo, hi = lp.var_lo.copy(), lp.var_hi.copy()
    two = np.isfinite(lo) & np.isfinite(hi) & (hi > lo)
    far_hi = two & (hi - x > 1e-3)
    far_lo = two & (x - lo > 1e-3) & ~far_hi
    hi[far_hi] = 1e9
    lo[far_lo] = -1e9
    wide = lpgen.LPData(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.vals, lp.c, lp.row_lo, lp.row_hi, lo, hi)
    st2, f2 = highs_solve(wide, sp, 0)
    if st2 != 0:
        return
    r2 = oracle_lib.solve(wide, sp, tol=1e-8, max_iter=400000, check_every=16, reduced_cost=1)
    assert r2.status[0] == 0
    assert abs(r2.obj[0] - f2) / (1 + abs(f2)) <= 1e-6


@pytest.mark.parametrize("seed", range(10))
def test_infeasibility_status_against_highs(oracle_lib, seed):
    lp = lpgen.random_lp(seed, 5, 7, feasible=False)
    sp = lpgen.base_specs(1)
    r = oracle_lib.solve(lp, sp, tol=1e-6, max_iter=200000, check_every=16)
    st, f = highs_solve(lp, sp, 0)
    want = {0: 0, 2: 1, 3: 2}[st]  # HiGHS optimal / infeasible / unbounded
    assert r.status[0] == want
    if want == 0:
        assert abs(r.obj[0] - f) / (1 + abs(f)) <= 1e-4


def test_hand_infeasible_and_unbounded(oracle_lib):
    lp = lpgen.from_dense([[1, 1]], [1, 1], [3], [INF], [0, 0], [1, 1])
    assert oracle_lib.solve(lp, lpgen.base_specs(1), tol=1e-6, check_every=16).status[0] == 1
    lp = lpgen.from_dense([[1, -1]], [-1, 0], [-INF], [1], [0, 0], [INF, INF])
    assert oracle_lib.solve(lp, lpgen.base_specs(1), tol=1e-6, check_every=16).status[0] == 2


def test_complementary_slackness_sign_of_y(oracle_lib):
    """y_i > 0 only on rows at their upper bound, y_i < 0 only at the lower
    bound (y in the barrier cone of [l,u], Sec. 3)."""
    w = lpgen.sb_small()
    r = oracle_lib.solve(w.lp, w.specs.subset([0]), tol=1e-9, max_iter=300000)
    x, y = r.x[0], r.y[0]
    ax = w.lp.matvec(x)
    scale = np.abs(y).max()
    up = y > 1e-5 * scale
    dn = y < -1e-5 * scale
    assert up.any() and dn.any()
    np.testing.assert_allclose(ax[up], w.lp.row_hi[up], atol=1e-5)
    np.testing.assert_allclose(ax[dn], w.lp.row_lo[dn], atol=1e-5)


def test_strong_branching_children_not_below_parent(oracle_lib):
    w = lpgen.sb_small()
    parent = oracle_lib.solve(w.lp, lpgen.base_specs(1), tol=1e-8, max_iter=200000)
    kids = oracle_lib.solve(w.lp, w.specs, tol=1e-8, max_iter=200000)
    assert np.all(kids.obj >= parent.obj[0] - 1e-6 * (1 + abs(parent.obj[0])))


def test_obbt_sandwich(oracle_lib):
    lp = lpgen.random_lp(5, 6, 8, density=0.5)
    cand = np.arange(lp.n)
    r = oracle_lib.solve(lp, lpgen.obbt_specs(cand), tol=1e-8, max_iter=400000, check_every=16)
    ok = r.status == 0
    lo, hi = r.obj[: lp.n], -r.obj[lp.n:]
    for j in range(lp.n):
        if ok[j]:
            assert lo[j] <= lp.x0[j] + 1e-5
            assert lo[j] >= lp.var_lo[j] - 1e-5
        if ok[lp.n + j]:
            assert hi[j] >= lp.x0[j] - 1e-5
            assert hi[j] <= lp.var_hi[j] + 1e-5


def test_batch_invariance_lockstep_vs_alone(oracle_lib):
    w = lpgen.sb_small()
    a = oracle_lib.solve(w.lp, w.specs, tol=1e-8, max_iter=200000, lockstep=1)
    b = oracle_lib.solve(w.lp, w.specs, tol=1e-8, max_iter=200000, lockstep=0, threads=4)
    np.testing.assert_array_equal(a.status, b.status)
    np.testing.assert_allclose(a.obj, b.obj, rtol=1e-6)


def test_threads_do_not_change_results(oracle_lib):
    w = lpgen.sb_small()
    a = oracle_lib.solve(w.lp, w.specs, tol=1e-6, max_iter=200000, threads=1)
    b = oracle_lib.solve(w.lp, w.specs, tol=1e-6, max_iter=200000, threads=4)
    np.testing.assert_array_equal(a.obj, b.obj)
    np.testing.assert_array_equal(a.iters, b.iters)


def test_empty_box_override_is_infeasible_at_zero_iterations(oracle_lib):
    w = lpgen.sb_small()
    sp = lpgen.make_specs([1, 0], [3, 0], [5.0, -INF], [4.0, INF])
    r = oracle_lib.solve(w.lp, sp, tol=1e-4, max_iter=100000)
    assert r.status[0] == 1 and r.iters[0] == 0
    assert r.status[1] == 0


def test_iteration_limit(oracle_lib):
    w = lpgen.sb_small()
    r = oracle_lib.solve(w.lp, w.specs.subset([0, 1]), tol=1e-12, max_iter=1)
    assert np.all(r.status == 3) and np.all(r.iters == 1)


def test_scaling_does_not_change_the_optimum(oracle_lib):
    w = lpgen.sb_small()
    sp = w.specs.subset([0, 9])
    a = oracle_lib.solve(w.lp, sp, tol=1e-8, max_iter=300000)
    b = oracle_lib.solve(w.lp, sp, tol=1e-8, max_iter=300000, ruiz_iters=0, pock_chambolle=0)
    np.testing.assert_allclose(a.obj, b.obj, rtol=1e-6)


# ---------------------------------------------------------------------------
# planted mistakes
# ---------------------------------------------------------------------------

def _pins_pass(o, mutation):
    """A fast subset of the pins; False as soon as one fails under `mutation`."""
    try:
        # hand KKT golden
        o.set_mutation(mutation)
        g = json.load(open(os.path.join(HERE, "golden", "kkt_handworked.json")))
        lpd = g["lp"]
        for case in g["cases"][:4]:
            lp = lpgen.from_dense(lpd["A"], lpd["c"], [_f(v) for v in lpd["row_lo"]],
                                  [_f(v) for v in lpd["row_hi"]], [_f(v) for v in case["var_lo"]],
                                  [_f(v) for v in case["var_hi"]])
            k = o.kkt(lp, 0, 0, 0.0, 0.0, 1.0, case["x"], case["y"])
            for key in ("obj", "dual_obj", "rel_primal", "rel_dual", "rel_gap"):
                if abs(k[key] - _f(case[key])) > 1e-12:
                    return False
        for case, lp in _robust_cases():
            k = o.kkt(lp, 0, 0, 0.0, 0.0, 1.0, case["x"], case["y"], reduced_cost=1)
            for key, v in case["modes"]["1"].items():
                if abs(k[key] - _f(v)) > 1e-12 * max(1.0, abs(_f(v))):
                    return False
        # nonexpansiveness on one LP
        lp, eta = _t_data(0)
        rng = np.random.default_rng(0)
        for w in (0.3, 4.0):
            for _ in range(30):
                z1 = rng.normal(size=lp.n) * 3, rng.normal(size=lp.m) * 3
                z2 = rng.normal(size=lp.n) * 3, rng.normal(size=lp.m) * 3
                t1 = o.apply_T(lp, lp.c, lp.var_lo, lp.var_hi, lp.row_lo, lp.row_hi, eta / w, eta * w, *z1)
                t2 = o.apply_T(lp, lp.c, lp.var_lo, lp.var_hi, lp.row_lo, lp.row_hi, eta / w, eta * w, *z2)
                if o.mnorm2(lp, w, eta, -1.0, t1[0] - t2[0], t1[1] - t2[1]) > \
                        o.mnorm2(lp, w, eta, -1.0, z1[0] - z2[0], z1[1] - z2[1]) * (1 + 1e-12) + 1e-12:
                    return False
        o.set_mutation(0)
        # the Halpern trajectory on a translation, with the mutation planted
        r = o.solve(_translation_lp(), lpgen.base_specs(1), tol=1e-12, max_iter=7, check_every=1,
                    detect_infeasibility=0, beta_s=0.0, beta_n=0.0, beta_a=1e9, warm_x=[0.5],
                    warm_y=np.zeros(0), mutation=mutation)
        if abs(r.x[0][0] - (0.5 - 7 * 0.998e-3)) > 1e-14:
            return False
        r = o.solve(lpgen.from_dense(np.ones((1, 1)), [0.0], [1.0], [np.inf], [0.0], [0.0]), lpgen.base_specs(1),
                    tol=1e-12, max_iter=7, check_every=1, detect_infeasibility=0, beta_s=0.0, beta_n=0.0,
                    beta_a=1e9, warm_x=[0.0], warm_y=[-0.25], mutation=mutation)
        if abs(r.y[0][0] - (-0.25 - 7 * 0.998)) > 1e-12:
            return False
        # the primal-weight update by hand, with the mutation planted
        lpw = lpgen.from_dense(np.array([[0.0, 1.0, 0.0]]), [0.3, 0.0, 0.4], [2.0], [INF], [-1e6, 0.0, 0.0],
                               [1e6, 0.0, 0.0])
        r = o.solve(lpw, lpgen.base_specs(1), tol=1e-12, max_iter=2, check_every=1, detect_infeasibility=0,
                    beta_s=1.0, beta_n=0.0, beta_a=1e9, warm_x=[0.0, 0.0, 0.0], warm_y=[0.0], mutation=mutation)
        w1 = math.sqrt((2 * 0.25 ** 2 / 0.3) * 0.25)
        if abs(r.x[0][0] + 0.3 * (0.998 / 0.25 + 0.998 / w1)) > 1e-9:
            return False
        # one Pock-Chambolle pass by hand, with the mutation planted
        o.set_mutation(mutation)
        for a, ruiz, dr_want, dc_want in handcases.pc_cases():
            lp = lpgen.from_dense(a, [1.0, 1.0], [-1.0, -1.0], [1.0, 1.0], [0.0, 0.0], [1.0, 1.0])
            dr, dc = o.scaling(lp, ruiz_iters=ruiz, pock_chambolle=True)
            if np.max(np.abs(dr - dr_want) / dr_want) > 1e-14 or np.max(np.abs(dc - dc_want) / dc_want) > 1e-14:
                return False
        o.set_mutation(0)
        # restart condition (ii) and the mean over active LPs by hand
        for beta_n, want in handcases.RESTART_BATCH_RESTARTS.items():
            if _restart_batch_solve(o, beta_n, mutation).restarts.tolist() != want:
                return False
        # HiGHS on two random LPs, through the solver with the mutation planted
        for seed in (1, 2):
            lp = lpgen.random_lp(seed, 5, 7)
            sp = lpgen.base_specs(1)
            r = o.solve(lp, sp, tol=1e-7, max_iter=30000, check_every=16, mutation=mutation)
            st, f = highs_solve(lp, sp, 0)
            if r.status[0] != 0 or abs(r.obj[0] - f) / (1 + abs(f)) > 1e-5:
                return False
        return True
    finally:
        o.set_mutation(0)


def test_pins_pass_without_mutation(oracle_lib):
    assert _pins_pass(oracle_lib, 0)


@pytest.mark.parametrize("mutation", range(1, 13))
def test_planted_mistakes_are_caught(oracle_lib, mutation):
    assert not _pins_pass(oracle_lib, mutation)
