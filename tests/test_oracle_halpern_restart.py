"""Pins for the evaluation step of the restarted reflected Halpern PDHG oracle
(Lu & Yang 2024, restarted Halpern PDHG; PDLP's restart tests and primal-weight
rule, Applegate et al. 2021).

At an evaluation with a restart the method must:
  * restart at the last map output z_hat = T(z_in), not at the Halpern iterate z:
    z = z0 = z_hat;
  * update the primal weight from the epoch's movement, dx = ||x_hat - x0||,
    dy = ||y_hat - y0||, by omega <- exp(0.5 ln(dy/dx) + 0.5 ln omega);
  * re-weight the new anchor value r_anchor with the NEW omega;
  * reset j and recompute tau = eta/omega, sigma = eta*omega.
Without a restart, r_prev takes the metric r and nothing else moves.  The
fixed-point-residual metric is r = sqrt(omega ||x_in - x_hat||^2 + ||y_in - y_hat||^2 / omega).

The states below are set by hand on a one-row LP with D_r = D_c = 1, so every
expected number is derived on paper from those definitions (the derivations
are in the comments), not by calling the oracle.  The last test plants each
plausible misreading into a copy of ``halpern_evaluate`` and checks that one
of these pins fails on it.
"""
import inspect
import math
import textwrap

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import lp as olp, pdhg, presolve as ops


def _one_row_lp():
    # min x1 + 2 x2  s.t.  x1 + x2 = 1,  0 <= x1 <= 10,  x2 >= 0 (no upper bound)
    lp = olp.LP(A=sp.csr_matrix(np.array([[1.0, 1.0]])), q=np.array([1.0]), c=np.array([1.0, 2.0]),
                l=np.array([0.0, 0.0]), u=np.array([10.0, np.inf]), m_eq=1)
    S = ops.scale(lp, ruiz_iters=0, pock_chambolle=False)
    assert np.all(S.Dr == 1.0) and np.all(S.Dc == 1.0)
    return S


def _state(S, metric, omega, r_anchor, r_prev, j, k):
    st = pdhg.halpern_initial_state(S, metric=metric)
    st.x0, st.y0 = np.array([0.0, 0.0]), np.array([0.0])          # epoch anchor z0
    st.xh, st.yh = np.array([3.0, 4.0]), np.array([20.0])         # last map output z_hat
    st.x_in, st.y_in = np.array([3.0, 7.0]), np.array([24.0])     # input of the last step
    st.x, st.y = np.array([1.0, 1.5]), np.array([5.0])            # Halpern iterate z
    st.omega, st.tau, st.sigma = omega, S.eta / omega, S.eta * omega
    st.r_anchor, st.r_prev, st.j, st.k, st.evals = r_anchor, r_prev, j, k, 0
    return st


# ||x_hat - x0|| = ||(3, 4)|| = 5, ||y_hat - y0|| = 20: from omega = 1 the rule
# gives exp(0.5 ln 4 + 0.5 ln 1) = 2.
# FPR parts: ||x_in - x_hat||^2 = 0 + 9 = 9, ||y_in - y_hat||^2 = 16.
# KKT of z_hat = ((3, 4), 20) on the unscaled LP:
#   r_p = 3 + 4 - 1 = 6                                   -> ||r_p||^2 = 36
#   lam = c - A^T y = (1 - 20, 2 - 20) = (-19, -18); x1 boxed: proj -19;
#   x2 only bounded below: proj max(-18, 0) = 0, r_d = (0, -18) -> ||r_d||^2 = 324
#   c.x = 3 + 8 = 11; dual obj = q.y + 10 min(-19, 0) = 20 - 190 = -170; gap = 181
#   KKT_w = sqrt(w^2 36 + 324 / w^2 + 181^2)
def _kkt_by_hand(w):
    return math.sqrt(w * w * 36.0 + 324.0 / (w * w) + 181.0 ** 2)


def _check_restart_fpr(evaluate):
    S = _one_row_lp()
    st = _state(S, "fpr", omega=1.0, r_anchor=100.0, r_prev=math.inf, j=10, k=64)
    status, _, _ = evaluate(S, st, pdhg._unscaled_lp(S), -1.0)
    assert status is None
    assert st.restarts == 1                                   # r = 5 <= 0.2 * 100
    assert st.omega == pytest.approx(2.0, rel=1e-14)
    np.testing.assert_array_equal(st.x, [3.0, 4.0])           # z = z_hat
    np.testing.assert_array_equal(st.y, [20.0])
    np.testing.assert_array_equal(st.x0, [3.0, 4.0])          # z0 = z_hat
    np.testing.assert_array_equal(st.y0, [20.0])
    assert st.r_anchor == pytest.approx(math.sqrt(2.0 * 9.0 + 16.0 / 2.0), rel=1e-14)   # new omega
    assert st.r_prev == math.inf
    assert st.j == 0
    assert st.tau == pytest.approx(S.eta / 2.0, rel=1e-15)
    assert st.sigma == pytest.approx(S.eta * 2.0, rel=1e-15)


def _check_restart_kkt(evaluate):
    S = _one_row_lp()
    st = _state(S, "kkt", omega=1.0, r_anchor=1e6, r_prev=math.inf, j=10, k=64)
    evaluate(S, st, pdhg._unscaled_lp(S), -1.0)
    assert st.restarts == 1                                   # KKT_1 = 182.0 <= 0.2e6
    assert st.omega == pytest.approx(2.0, rel=1e-14)
    np.testing.assert_array_equal(st.x0, [3.0, 4.0])
    np.testing.assert_array_equal(st.y0, [20.0])
    assert st.r_anchor == pytest.approx(_kkt_by_hand(2.0), rel=1e-14)
    assert st.r_anchor != pytest.approx(_kkt_by_hand(1.0), rel=1e-6)   # the old weight would differ


def _check_no_restart(evaluate):
    S = _one_row_lp()
    # omega = 4: r = sqrt(4 * 9 + 16 / 4) = sqrt(40) = 6.32 > 0.8 * 5.5, j = 10 < 0.36 * 64
    st = _state(S, "fpr", omega=4.0, r_anchor=5.5, r_prev=math.inf, j=10, k=64)
    evaluate(S, st, pdhg._unscaled_lp(S), -1.0)
    assert st.restarts == 0
    assert st.r_prev == pytest.approx(math.sqrt(40.0), rel=1e-15)
    assert st.omega == 4.0 and st.r_anchor == 5.5 and st.j == 10
    np.testing.assert_array_equal(st.x, [1.0, 1.5])
    np.testing.assert_array_equal(st.x0, [0.0, 0.0])
    # the KKT metric without a restart: r_prev = KKT_4(z_hat)
    st = _state(S, "kkt", omega=4.0, r_anchor=200.0, r_prev=math.inf, j=10, k=64)
    evaluate(S, st, pdhg._unscaled_lp(S), -1.0)
    assert st.restarts == 0
    assert st.r_prev == pytest.approx(_kkt_by_hand(4.0), rel=1e-14)


def _check_restart_lands_on_fixed_point(evaluate):
    # a box LP whose only row is slack: T maps every point of the box to its
    # fixed point z* = ((0, 1, 0), 0) in one step.  The Halpern iterate is pulled
    # toward z0 = 0 (z_j = z* - z*/(j+1)), so only a restart at z_hat = z* lands
    # on the fixed point; from there every later step stays on it exactly.
    lp = olp.LP(A=sp.csr_matrix(np.array([[1.0, 1.0, 1.0]])), q=np.array([-100.0]),
                c=np.array([1.0, -1.0, 2.0]), l=np.zeros(3), u=np.array([1.0, 1.0, 5.0]), m_eq=0)
    S = ops.scale(lp, ruiz_iters=0, pock_chambolle=False)
    U = pdhg._unscaled_lp(S)
    st = pdhg.halpern_initial_state(S)
    AT = S.A.T.tocsr()
    for _ in range(pdhg.N_EVAL):
        pdhg.halpern_step(S, st, AT)
    assert not np.array_equal(st.x, [0.0, 1.0, 0.0])          # the iterate is not z* yet
    evaluate(S, st, U, -1.0)                                  # j = 64 >= 0.36 * 64: restart
    assert st.restarts == 1
    for _ in range(10):
        np.testing.assert_array_equal(st.x, [0.0, 1.0, 0.0])
        np.testing.assert_array_equal(st.y, [0.0])
        pdhg.halpern_step(S, st, AT)


# The PDHG-norm residual ("fprp"): dx = x_in - x_hat = (0, 3), dy = y_in - y_hat = 4,
# A dx = 3, so dy.A dx = 12; without scaling eta = 0.998 / sqrt(||A||_1 ||A||_inf)
# = 0.998 / sqrt(2).  r_omega = sqrt(omega 9 + 16 / omega - 24 eta).
def _check_fprp(evaluate):
    S = _one_row_lp()
    eta = 0.998 / math.sqrt(2.0)
    assert S.eta == pytest.approx(eta, rel=1e-15)
    st = _state(S, "fprp", omega=4.0, r_anchor=5.0, r_prev=math.inf, j=10, k=64)
    evaluate(S, st, pdhg._unscaled_lp(S), -1.0)
    assert st.restarts == 0
    assert st.r_prev == pytest.approx(math.sqrt(36.0 + 4.0 - 24.0 * eta), rel=1e-14)
    st = _state(S, "fprp", omega=1.0, r_anchor=100.0, r_prev=math.inf, j=10, k=64)
    evaluate(S, st, pdhg._unscaled_lp(S), -1.0)
    assert st.restarts == 1 and st.omega == pytest.approx(2.0, rel=1e-14)
    assert st.r_anchor == pytest.approx(math.sqrt(18.0 + 8.0 - 24.0 * eta), rel=1e-14)


# The residual-balance guard on the weight update.  At z_hat the relative
# residuals are rel_p = 6 / (1 + |q|) = 3 and rel_d = 18 / (1 + |c|_inf) = 6: the
# dual residual leads, so an increase of omega (toward a larger dual step,
# which works on the primal residual) is dropped once rel_d > kappa rel_p, and a
# decrease is never dropped.
def _check_guard(evaluate):
    S = _one_row_lp()
    # kappa = 1: 1 -> 2 would widen the imbalance (6 > 1 * 3): omega stays 1 and
    # the anchor value, the steps and the restart itself use omega = 1
    st = _state(S, "kkt", omega=1.0, r_anchor=1e6, r_prev=math.inf, j=10, k=64)
    st.pw_guard = 1.0
    evaluate(S, st, pdhg._unscaled_lp(S), -1.0)
    assert st.restarts == 1 and st.omega == 1.0
    assert st.r_anchor == pytest.approx(_kkt_by_hand(1.0), rel=1e-14)
    assert st.tau == pytest.approx(S.eta, rel=1e-15) and st.j == 0
    np.testing.assert_array_equal(st.x0, [3.0, 4.0])
    # kappa = 2: 6 > 2 * 3 is false, the update stands
    st = _state(S, "kkt", omega=1.0, r_anchor=1e6, r_prev=math.inf, j=10, k=64)
    st.pw_guard = 2.0
    evaluate(S, st, pdhg._unscaled_lp(S), -1.0)
    assert st.omega == pytest.approx(2.0, rel=1e-14)
    # a decrease, 16 -> exp(0.5 ln 4 + 0.5 ln 16) = 8, moves toward balance: kept
    # (KKT_16 = sqrt(256 * 36 + 324 / 256 + 181^2) = 204.9 <= 0.2e6: a restart)
    st = _state(S, "kkt", omega=16.0, r_anchor=1e6, r_prev=math.inf, j=10, k=64)
    st.pw_guard = 1.0
    evaluate(S, st, pdhg._unscaled_lp(S), -1.0)
    assert st.restarts == 1 and st.omega == pytest.approx(8.0, rel=1e-14)
    # guard off: the plain update
    st = _state(S, "kkt", omega=1.0, r_anchor=1e6, r_prev=math.inf, j=10, k=64)
    evaluate(S, st, pdhg._unscaled_lp(S), -1.0)
    assert st.omega == pytest.approx(2.0, rel=1e-14)


PINS = [_check_restart_fpr, _check_restart_kkt, _check_no_restart, _check_restart_lands_on_fixed_point,
        _check_fprp, _check_guard]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__[7:])
def test_halpern_evaluate_pins(pin):
    pin(pdhg.halpern_evaluate)


MUTANTS = {
    "restart at the Halpern iterate z": [("st.x = st.xh.copy()", "st.x = st.x.copy()"),
                                         ("st.y = st.yh.copy()", "st.y = st.y.copy()")],
    "movement measured from z, not z0": [("np.linalg.norm(st.xh - st.x0)", "np.linalg.norm(st.xh - st.x)")],
    "movement measured from the step input": [("np.linalg.norm(st.yh - st.y0)", "np.linalg.norm(st.yh - st.y_in)")],
    "anchor value with the old weight (kkt)": [("parts[2], wn)", "parts[2], w)")],
    "anchor value with the old weight (fpr)": [("max(wn * fx2 + fy2 / wn", "max(w * fx2 + fy2 / w")],
    "weight on the wrong block of the residual": [("max(w * fx2 + fy2 / w", "max(fx2 / w + w * fy2")],
    "cross term of the PDHG norm dropped": [("cross = float(np.dot(", "cross = 0.0 * float(np.dot(")],
    "cross term with the wrong sign": [("fy2 / w - 2.0 * S.eta * cross", "fy2 / w + 2.0 * S.eta * cross")],
    "r_prev left unchanged": [("st.r_prev = r\n", "st.r_prev = st.r_prev\n")],
    "j not reset": [("st.j = 0", "st.j = st.j")],
    "primal weight rule inverted": [("primal_weight_update(w, dx, dy, st.pw)", "primal_weight_update(w, dy, dx, st.pw)")],
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_each_planted_mistake_fails_a_pin(name):
    fn = pdhg.halpern_evaluate
    src = textwrap.dedent(inspect.getsource(fn))
    for old, new in MUTANTS[name]:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    ns = dict(vars(pdhg))
    exec(compile(src, "<mutant>", "exec"), ns)
    bad = ns["halpern_evaluate"]
    failed = []
    for pin in PINS:
        try:
            pin(bad)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"no pin caught the planted mistake: {name}"


GUARD_MUTANTS = {
    "guard directions swapped": [("omega_new < omega and rel_p", "omega_new > omega and rel_p"),
                                 ("omega_new > omega and rel_d", "omega_new < omega and rel_d")],
    "guard compares the residuals the wrong way": [("rel_d > kappa * rel_p", "rel_p > kappa * rel_d")],
    "guard with a non-strict comparison": [("rel_d > kappa * rel_p", "rel_d >= kappa * rel_p")],
    "guard without the factor kappa": [("rel_d > kappa * rel_p", "rel_d > rel_p")],
    "guard always on": [("if kappa > 0.0 and (", "if kappa >= 0.0 and (")],
}


@pytest.mark.parametrize("name", sorted(GUARD_MUTANTS))
def test_each_planted_guard_mistake_fails_the_guard_pin(name):
    src = textwrap.dedent(inspect.getsource(pdhg.guard_weight))
    for old, new in GUARD_MUTANTS[name]:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    ns = dict(vars(pdhg))
    exec(compile(src, "<mutant>", "exec"), ns)
    # halpern_evaluate compiled in the same namespace calls the planted guard
    exec(compile(textwrap.dedent(inspect.getsource(pdhg.halpern_evaluate)), "<mutant>", "exec"), ns)
    with pytest.raises(AssertionError):
        _check_guard(ns["halpern_evaluate"])
