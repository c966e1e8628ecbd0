"""Small LPs whose behaviour under the method is derived by hand, shared by
the oracle pins (CPU) and the GPU tests.  Only data and hand-derived
expectations live here; no step of the method is computed.

restart_batch(): Sec. 4 "Restarts" and Sec. 5 "Restarts" (the batch-averaged
residual, reading R11: the mean over the LPs still active at the check) on a
lockstep batch of five LPs with n = 2, no rows.

  With no rows, ||A~|| = 0 gives eta = 0.998 and every primal weight stays
  w = 1 (readings R2, R3; the weight update needs ||dy0|| > 0), so
  tau = 0.998.  An LP whose variable moves in the interior is a translation
  T(z) = z - tau c, so the Halpern iterate is z^k = z^0 - k tau c and its
  residual at every check is r = sqrt(w/eta) |tau c| = sqrt(eta) |c|;
  restarting a translation at T(z) continues the same line.  Checks follow
  every iteration; check K (0-based) evaluates T(z^K).

  base c = (1/8, 0), x1 in [-1000, 1000], x2 in [-2.5, 5.5], z^0 = 0:
    P1, P2  base LP: x1 moves down by 0.12475 forever; r = sqrt(eta)/8.
    R       x1 >= -0.4375: x1 - 0.12475 k meets the bound at check 3
            (0.37425 + 0.12475 > 0.4375), where T(z) is the optimum: it
            finishes there (4 iterations); r = sqrt(eta)/8 before.
    B1      min x2: x2 moves down by 0.998 and finishes at check 2 (x2 = -2.5).
    B2      max x2: x2 moves up by 0.998 and finishes at check 5 (x2 = 5.5).
            B1 and B2 have c = +-e_2, so r = sqrt(eta) before they finish.
  In units of sqrt(eta), the mean over the active LPs (finished LPs leave
  at the check where they finish) is
    checks 0-1: (3/8 + 2)/5 = 0.475 (r0, set at check 0)
    check  2:   (3/8 + 1)/4 = 0.34375   (0.7237 r0, a decrease)
    checks 3-4: (2/8 + 1)/3 = 0.41667   (0.8772 r0, an increase)
    checks 5-6: 2/8 / 2     = 0.125
  The decrease and the increase come at consecutive checks, and every
  repeated value sits above beta_n r0, so rounding noise between equal
  values can never meet condition (ii).  With beta_s = 0.2 and
  beta_a = 1e9 (no artificial restarts), 7 iterations (the last check ends
  the solve without a restart test):
    beta_n = 0.9: condition (ii) (r <= beta_n r0 and r > r_prev) restarts at
      check 3; r0 becomes 0.41667 and check 5 sees 0.3 r0, above beta_s and a
      decrease: one restart.  (With "r < r_prev" it would restart at checks
      2 and 5.)
    beta_n = 0.5: nothing restarts (0.8772 > 0.5; 0.125 / 0.475 = 0.263 is
      above beta_s and a decrease): zero restarts.  (Without the beta_n
      clause check 3 would restart; dividing by all five LPs instead of the
      active ones gives 0.05 / 0.475 = 0.105 <= beta_s at check 5.)
  P1 and P2 end at the iteration limit.

pc_cases(): one Pock-Chambolle pass (alpha = 1, reading R1) on a 2 x 2
matrix, alone and after one Ruiz pass, with factors written out by hand.
"""
import math

import numpy as np

import lpgen

INF = np.inf


def restart_batch():
    lp = lpgen.from_dense(np.zeros((0, 2)), [0.125, 0.0], [], [], [-1000.0, -2.5], [1000.0, 5.5])
    specs = lpgen.make_specs(kind=[0, 0, 1, 2, 2], var=[0, 0, 0, 1, 1],
                             lo=[-INF, -INF, -0.4375, -INF, -INF], hi=[INF, INF, INF, INF, INF],
                             sign=[1.0, 1.0, 1.0, 1.0, -1.0], label=["P1", "P2", "R", "B1", "B2"])
    warm_x = np.zeros((5, 2))
    warm_y = np.zeros((5, 0))
    return lp, specs, warm_x, warm_y


RESTART_BATCH_MAX_ITER = 7
RESTART_BATCH_ITERS = [7, 7, 4, 3, 6]          # per LP: finishing iteration (7 = the limit)
RESTART_BATCH_STATUS = [3, 3, 0, 0, 0]         # ITERATION_LIMIT for P1, P2; OPTIMAL otherwise
RESTART_BATCH_OPT_X = {2: (-0.4375, 0.0), 3: (0.0, -2.5), 4: (0.0, 5.5)}
# beta_n -> restarts per LP: the restart at check 3 counts for the LPs still
# active after it (P1, P2, B2; R finishes at check 3 before the restart test)
RESTART_BATCH_RESTARTS = {0.9: [1, 1, 0, 0, 1], 0.5: [0, 0, 0, 0, 0]}
RESTART_BATCH_KW = dict(check_every=1, detect_infeasibility=0, beta_s=0.2, beta_a=1e9)


def pc_cases():
    """(A, ruiz_iters, D_r, D_c) with A~ = D_r A D_c after the passes."""
    a = np.array([[1.0, 3.0], [2.0, 4.0]])
    # Pock-Chambolle alone: row sums 4, 6; column sums 3, 7
    pc_only = (a, 0, np.array([1 / 2, 1 / math.sqrt(6)]), np.array([1 / math.sqrt(3), 1 / math.sqrt(7)]))
    # one Ruiz pass: row inf-norms 3, 4, column inf-norms 2, 4 give
    # D_r = (1/sqrt 3, 1/2), D_c = (1/sqrt 2, 1/2) and
    # A~ = [[1/sqrt 6, sqrt(3)/2], [1/sqrt 2, 1]]; then Pock-Chambolle divides
    # by the square roots of A~'s row and column sums
    rho = (1 / math.sqrt(6) + math.sqrt(3) / 2, 1 / math.sqrt(2) + 1.0)
    kap = (1 / math.sqrt(6) + 1 / math.sqrt(2), math.sqrt(3) / 2 + 1.0)
    ruiz_pc = (a, 1, np.array([1 / math.sqrt(3) / math.sqrt(rho[0]), 0.5 / math.sqrt(rho[1])]),
               np.array([1 / math.sqrt(2) / math.sqrt(kap[0]), 0.5 / math.sqrt(kap[1])]))
    return [pc_only, ruiz_pc]
