"""The iteration's restart logic on the GPU against values derived by hand
(tests/handcases.py and the oracle pins that use the same cases): restart
condition (ii) with the batch mean over active LPs, the artificial and
sufficient-decay restart schedule, one primal-weight update, and one
Pock-Chambolle pass.  Each case runs through the C ABI in FP64 and in mixed
precision (FP32 iterates, double-float checks)."""
import math

import numpy as np
import pytest

import handcases
import lpgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lpb():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2601_21990_gb300 import _build, lpb as mod

    _build.build()
    mod.load()
    return mod


def _prec(lpb, precision):
    return lpb.FP64 if precision == "fp64" else lpb.MIXED


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_restart_condition_ii_and_active_mean(lpb, precision):
    """Five LPs in one batch (one restart group): the mean residual over the
    LPs still active falls at check 2 and rises at check 3 below beta_n r0,
    so condition (ii) restarts once at check 3 for beta_n = 0.9 and never for
    beta_n = 0.5; statuses, finishing iterations, per-LP restart counts and
    the finished LPs' optima as derived by hand."""
    lp, specs, wx, wy = handcases.restart_batch()
    for beta_n, want in handcases.RESTART_BATCH_RESTARTS.items():
        h = lpb.Handle(lp, precision=_prec(lpb, precision), fp64_polish=0, beta_n=beta_n,
                       **handcases.RESTART_BATCH_KW)
        assert h.info()[0] == 0.998
        b = h.solve(specs, tol=1e-12, max_iter=handcases.RESTART_BATCH_MAX_ITER, warm_x=wx.ravel(),
                    warm_y=wy.ravel())
        res = b.results()
        assert res["status"].tolist() == handcases.RESTART_BATCH_STATUS, (beta_n, res["status"])
        assert res["iters"].tolist() == handcases.RESTART_BATCH_ITERS, (beta_n, res["iters"])
        assert res["restarts"].tolist() == want, (beta_n, res["restarts"])
        for q, xq in handcases.RESTART_BATCH_OPT_X.items():
            r, x, y = b.result(q)
            np.testing.assert_allclose(x, xq, atol=1e-15)
        b.free()
        h.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_restart_schedule_by_hand(lpb, precision):
    """Sec. 4 "Restarts" in reading R5 on the translation LP (one variable, no
    rows, cost 1e-3), whose residual is the same at every check: checks
    every 4 iterations over 72 iterations restart 5 times by the artificial
    condition k > 0.36 K alone, and 17 times with beta_s = 1 (every check but
    the last); the point stays z0 - 72 delta."""
    lp = lpgen.from_dense(np.zeros((0, 1)), [1e-3], [], [], [-1.0], [1.0])
    for kw, want in ((dict(beta_s=0.0, beta_n=0.0, beta_a=0.36), 5), (dict(beta_s=1.0, beta_n=0.0, beta_a=1e9), 17)):
        h = lpb.Handle(lp, precision=_prec(lpb, precision), check_every=4, detect_infeasibility=0, fp64_polish=0,
                       **kw)
        b = h.solve(lpgen.base_specs(1), tol=1e-12, max_iter=72, warm_x=np.array([0.5]))
        r, x, y = b.result(0)
        assert r.status == lpb.ITERATION_LIMIT and r.iters == 72
        assert r.restarts == want, kw
        assert x[0] == pytest.approx(0.5 - 72 * 0.998e-3, abs=1e-14 if precision == "fp64" else 1e-5)
        b.free()
        h.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_primal_weight_update_by_hand(lpb, precision):
    """Sec. 4 "Step-size and primal weight" (readings R3, R7): x1 free with
    cost 0.3, x2 fixed at 0 under the row x2 >= 2 (infeasible, detection
    off), x3 fixed with cost 0.4; eta = 0.998, w0 = 0.5 / 2.  The first
    check restarts (beta_s = 1) with d = ||dy|| / ||dx|| = 2 w0^2 / c1 and
    w1 = sqrt(d w0); the second iteration steps with tau1 = eta / w1,
    sigma1 = eta w1, so x1 = -c1 (tau0 + tau1) and y = -2 (sigma0 + sigma1)."""
    inf = np.inf
    lp = lpgen.from_dense(np.array([[0.0, 1.0, 0.0]]), [0.3, 0.0, 0.4], [2.0], [inf], [-1e6, 0.0, 0.0],
                          [1e6, 0.0, 0.0])
    eta, c1, w0 = 0.998, 0.3, 0.25
    w1 = math.exp(0.5 * math.log(2 * w0 ** 2 / c1) + 0.5 * math.log(w0))
    h = lpb.Handle(lp, precision=_prec(lpb, precision), check_every=1, detect_infeasibility=0, beta_s=1.0,
                   beta_n=0.0, beta_a=1e9, fp64_polish=0)
    assert h.info()[0] == pytest.approx(eta, rel=1e-12)
    b = h.solve(lpgen.base_specs(1), tol=1e-12, max_iter=2, warm_x=np.zeros(3), warm_y=np.zeros(1))
    r, x, y = b.result(0)
    assert r.status == lpb.ITERATION_LIMIT and r.iters == 2 and r.restarts == 1
    rel = 1e-12 if precision == "fp64" else 2e-6
    assert x[0] == pytest.approx(-c1 * (eta / w0 + eta / w1), rel=rel)
    assert y[0] == pytest.approx(-2 * (eta * w0 + eta * w1), rel=rel)
    # the printed ratio ||dx|| / ||dy|| would give x1 = -1.584 instead of -2.125
    assert abs(x[0] + 1.584) > 0.1
    b.free()
    h.close()


def test_pock_chambolle_pass_by_hand(lpb):
    """Reading R1's Pock-Chambolle pass on a 2 x 2 matrix, alone and after
    one Ruiz pass: the factors lpb_create computes against the hand values."""
    for a, ruiz, dr_want, dc_want in handcases.pc_cases():
        lp = lpgen.from_dense(a, [1.0, 1.0], [-1.0, -1.0], [1.0, 1.0], [0.0, 0.0], [1.0, 1.0])
        h = lpb.Handle(lp, precision=lpb.FP64, ruiz_iters=ruiz, pock_chambolle=1)
        dr, dc = h.scaling()
        np.testing.assert_allclose(dr, dr_want, rtol=1e-14)
        np.testing.assert_allclose(dc, dc_want, rtol=1e-14)
        h.close()
