"""Pins for O1 (FP64 restarted PDHG): convergence to the simplex optimum,
closed-form fixed points, step invariants and the restart rules."""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import ucgen
from oracle import kkt, lp as olp, pdhg, presolve as ops, simplex

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _pipeline(P):
    raw = olp.build_lp(P)
    ps = ops.presolve(raw)
    S = ops.scale(ps.lp)
    return raw, ps, S


@pytest.mark.parametrize("seed", range(3))
def test_pdhg_reaches_simplex_objective(seed):
    P = ucgen.make_problem(seed, B=12, L=16, G=4, T=6, lo=0.4, hi=0.8, noise=0.05,
                           zero_pmin_frac=0.25)
    raw, ps, S = _pipeline(P)
    r = pdhg.solve(S, tol=1e-4, max_iter=100_000)
    assert r.status == "optimal"
    x = S.Dc * r.x
    y = S.Dr * r.y
    assert max(kkt.relative_kkt(ps.lp, x, y)) <= 1e-4       # independent KKT evaluation
    ref = simplex.solve_lp(raw)
    xr, _ = ops.postsolve(ps, x)
    obj = float(raw.c @ xr)
    assert abs(obj - ref.obj) / max(1.0, abs(ref.obj)) <= 1e-4


def test_pdhg_tiny_objective_matches_golden():
    with open(os.path.join(GOLDEN, "tiny_lp.json")) as f:
        g = json.load(f)
    P = ucgen.tiny(g["seed"])
    raw, ps, S = _pipeline(P)
    r = pdhg.solve(S, tol=1e-4, max_iter=100_000)
    assert r.status == "optimal"
    xr, _ = ops.postsolve(ps, S.Dc * r.x)
    obj = float(raw.c @ xr)
    assert abs(obj - g["objective"]) / abs(g["objective"]) <= 1e-4


def test_pdhg_iterates_stay_in_their_sets():
    P = ucgen.micro(0, B=10, L=13, G=4, T=6)
    raw, ps, S = _pipeline(P)
    st = pdhg.initial_state(S)
    U = pdhg._unscaled_lp(S)
    AT = S.A.T.tocsr()
    for _ in range(300):
        pdhg.step(S, st, AT)
        assert np.all(st.x >= S.l) and np.all(st.x <= S.u)
        assert np.all(st.y[S.m_eq:] >= 0.0)
        if st.k % pdhg.N_EVAL == 0:
            pdhg.evaluate(S, st, U, 0.0)
            assert np.all(st.x >= S.l) and np.all(st.x <= S.u)


def test_pdhg_box_minimiser_in_one_step():
    # the only row is slack everywhere in the box, so the LP optimum is the
    # box-clipped minimiser of c.x, reached by the first primal step
    lp = olp.LP(A=sp.csr_matrix(np.array([[1.0, 1.0, 1.0]])), q=np.array([-100.0]),
                c=np.array([1.0, -1.0, 2.0]), l=np.zeros(3), u=np.array([1.0, 1.0, 5.0]), m_eq=0)
    S = ops.scale(lp, ruiz_iters=0, pock_chambolle=False)
    st = pdhg.initial_state(S)
    assert st.tau * np.min(np.abs(S.c)) >= np.max(S.u - S.l)
    pdhg.step(S, st)
    np.testing.assert_array_equal(st.x, [0.0, 1.0, 0.0])
    np.testing.assert_array_equal(st.y, [0.0])
    r = pdhg.solve(S, tol=1e-12, max_iter=1000)
    assert r.status == "optimal" and r.iters == pdhg.N_EVAL


def test_pdhg_single_equality_row_fixed_point():
    # min c.x s.t. a.x = b, 0 <= x <= 1: fill columns in increasing c_j / a_j
    a = np.array([1.0, 2.0, 0.5, 1.5, 1.0])
    c = np.array([3.0, 2.0, 4.0, 1.0, 6.0])
    b = 2.7
    order = np.argsort(c / a)
    xs = np.zeros(5)
    left = b
    for j in order:
        xs[j] = min(1.0, left / a[j])
        left -= a[j] * xs[j]
        if left <= 0:
            break
    lp = olp.LP(A=sp.csr_matrix(a[None, :]), q=np.array([b]), c=c, l=np.zeros(5),
                u=np.ones(5), m_eq=1)
    S = ops.scale(lp)
    r = pdhg.solve(S, tol=1e-9, max_iter=200_000)
    assert r.status == "optimal"
    np.testing.assert_allclose(S.Dc * r.x, xs, atol=1e-6)
    mu = c[order][np.searchsorted(np.cumsum(a[order]), b)] / a[order][np.searchsorted(np.cumsum(a[order]), b)]
    assert abs(S.Dr[0] * r.y[0] - mu) <= 1e-6 * mu          # the row's price is the marginal ratio


def test_restart_rules_scripted():
    inf = math.inf
    assert pdhg.restart_decision(0.19, 1.0, inf, 10, 1000)        # sufficient decay
    assert not pdhg.restart_decision(0.21, 1.0, inf, 10, 1000)
    assert pdhg.restart_decision(0.5, 1.0, 0.4, 10, 1000)         # necessary decay, no progress
    assert not pdhg.restart_decision(0.5, 1.0, 0.6, 10, 1000)     # still improving
    assert not pdhg.restart_decision(0.9, 1.0, 0.6, 10, 1000)     # not decayed enough
    assert pdhg.restart_decision(0.9, 1.0, 0.6, 360, 1000)        # long epoch (artificial)
    assert not pdhg.restart_decision(0.9, 1.0, 0.6, 359, 1000)


def test_primal_weight_rule_scripted():
    assert pdhg.primal_weight_update(1.0, 1.0, 4.0) == pytest.approx(2.0, rel=1e-15)
    assert pdhg.primal_weight_update(4.0, 2.0, 2.0) == pytest.approx(2.0, rel=1e-15)
    assert pdhg.primal_weight_update(3.0, 0.0, 1.0) == 3.0         # movement too small: keep
    assert pdhg.primal_weight_update(3.0, 1.0, 1e-11) == 3.0


def test_primal_weight_controller_by_hand():
    # e = ln(omega dx / dy); ln omega <- ln omega - (kp e + ki sum e + kd (e - e_prev))
    ctl = pdhg.PrimalWeightControl(kp=0.3, ki=0.02, kd=0.3)
    # omega = 1, dx = 1, dy = e^2: e1 = -2, no derivative yet: ln omega = 2 (0.3 + 0.02) = 0.64
    w1 = pdhg.primal_weight_update(1.0, 1.0, math.exp(2.0), ctl)
    assert w1 == pytest.approx(math.exp(0.64), rel=1e-14)
    # dx = 1, dy = e^0.64 * e^1: e2 = 0.64 - 1.64 = -1, sum = -3, de = +1:
    # ln omega = 0.64 - (-0.3 - 0.06 + 0.3) = 0.70
    w2 = pdhg.primal_weight_update(w1, 1.0, math.exp(1.64), ctl)
    assert w2 == pytest.approx(math.exp(0.70), rel=1e-14)
    # a step with no movement keeps omega and the controller's state
    assert pdhg.primal_weight_update(w2, 0.0, 1.0, ctl) == w2 and ctl.isum == pytest.approx(-3.0)


@pytest.mark.parametrize("gains", [pdhg.PDLP_GAINS, pdhg.DEFAULT_PW_GAINS, (0.3, 0.02, 0.3)])
def test_primal_weight_controller_settles_on_the_balance(gains):
    # a plant whose movement ratio dy/dx = rho does not depend on omega: the
    # controller's only rest point has e = 0, i.e. omega = rho
    for rho in (1e-3, 0.7, 250.0):
        ctl = pdhg.PrimalWeightControl(*gains)
        w = 1.0
        for _ in range(200):
            w = pdhg.primal_weight_update(w, 1.0, rho, ctl)
        assert abs(math.log(w / rho)) <= 1e-6, (gains, rho, w)


def test_first_evaluation_restarts():
    P = ucgen.micro(1, B=6, L=8, G=3, T=4)
    raw, ps, S = _pipeline(P)
    seen = {}
    pdhg.solve(S, tol=0.0, max_iter=pdhg.N_EVAL,
               trace=lambda k, st: seen.setdefault(k, (st.restarts, st.j)), trace_iters=[pdhg.N_EVAL])
    assert seen[pdhg.N_EVAL] == (1, 0)       # j = 64 >= 0.36 * 64 always fires


# ---------------------------------------------------------------------------
# Halpern variant (the default)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("metric", ["kkt", "fpr", "fprp"])
@pytest.mark.parametrize("seed", range(3))
def test_halpern_reaches_simplex_objective(seed, metric):
    P = ucgen.make_problem(seed, B=12, L=16, G=4, T=6, lo=0.4, hi=0.8, noise=0.05,
                           zero_pmin_frac=0.25)
    raw, ps, S = _pipeline(P)
    r = pdhg.solve_halpern(S, tol=1e-4, max_iter=100_000, metric=metric)
    assert r.status == "optimal"
    x, y = S.Dc * r.x, S.Dr * r.y
    assert max(kkt.relative_kkt(ps.lp, x, y)) <= 1e-4
    ref = simplex.solve_lp(raw)
    xr, _ = ops.postsolve(ps, x)
    assert abs(float(raw.c @ xr) - ref.obj) / max(1.0, abs(ref.obj)) <= 1e-4


def test_halpern_tiny_objective_matches_golden():
    with open(os.path.join(GOLDEN, "tiny_lp.json")) as f:
        g = json.load(f)
    raw, ps, S = _pipeline(ucgen.tiny(g["seed"]))
    r = pdhg.solve_halpern(S, tol=1e-4)
    assert r.status == "optimal"
    xr, _ = ops.postsolve(ps, S.Dc * r.x)
    assert abs(float(raw.c @ xr) - g["objective"]) / abs(g["objective"]) <= 1e-4


def test_halpern_first_step_is_the_pdhg_step_and_maps_stay_feasible():
    raw, ps, S = _pipeline(ucgen.micro(0, B=10, L=13, G=4, T=6))
    st_p = pdhg.initial_state(S)
    st_h = pdhg.halpern_initial_state(S)
    pdhg.step(S, st_p)
    pdhg.halpern_step(S, st_h)
    # w = 1/2 on the first step of an epoch: z1 = (2 T(z0) - z0)/2 + z0/2 = T(z0)
    np.testing.assert_allclose(st_h.x, st_p.x, rtol=0, atol=1e-12)
    np.testing.assert_allclose(st_h.y, st_p.y, rtol=0, atol=1e-12)
    U = pdhg._unscaled_lp(S)
    for _ in range(300):
        pdhg.halpern_step(S, st_h)
        assert np.all(st_h.xh >= S.l) and np.all(st_h.xh <= S.u)
        assert np.all(st_h.yh[S.m_eq:] >= 0.0)
        if st_h.k % pdhg.N_EVAL == 0:
            pdhg.halpern_evaluate(S, st_h, U, 0.0)


def test_halpern_second_step_weight():
    # with no active constraint the map reaches its fixed point in one step; the
    # second step's weight w = 2/3 then pulls z back toward the anchor z0 = 0
    lp = olp.LP(A=sp.csr_matrix(np.array([[1.0, 1.0, 1.0]])), q=np.array([-100.0]),
                c=np.array([1.0, -1.0, 2.0]), l=np.zeros(3), u=np.array([1.0, 1.0, 5.0]), m_eq=0)
    S = ops.scale(lp, ruiz_iters=0, pock_chambolle=False)
    st = pdhg.halpern_initial_state(S)
    pdhg.halpern_step(S, st)
    pdhg.halpern_step(S, st)
    # z2 = 2/3 (2 T(z1) - z1) + 1/3 z0 with T(z1) = z1 = (0, 1, 0), z0 = 0
    np.testing.assert_allclose(st.x, [0.0, 2.0 / 3.0, 0.0], rtol=0, atol=1e-15)


# ---------------------------------------------------------------------------
# adaptive step size (PDLP, averaging variant)
# ---------------------------------------------------------------------------
def _small(seed):
    return ucgen.make_problem(seed, B=12, L=16, G=4, T=6, lo=0.4, hi=0.8, noise=0.05, zero_pmin_frac=0.25)


@pytest.mark.parametrize("seed", range(3))
def test_adaptive_reaches_simplex_objective(seed):
    raw, ps, S = _pipeline(_small(seed))
    att = []
    r = pdhg.solve(S, tol=1e-4, max_iter=100_000, adaptive=True, attempts=att)
    assert r.status == "optimal"
    assert any(not a[0] for a in att), "the rule never rejected a step"
    x, y = S.Dc * r.x, S.Dr * r.y
    assert max(kkt.relative_kkt(ps.lp, x, y)) <= 1e-4
    ref = simplex.solve_lp(raw)
    xr, _ = ops.postsolve(ps, x)
    assert abs(float(raw.c @ xr) - ref.obj) / max(1.0, abs(ref.obj)) <= 1e-4


def test_adaptive_tiny_objective_matches_golden():
    with open(os.path.join(GOLDEN, "tiny_lp.json")) as f:
        g = json.load(f)
    raw, ps, S = _pipeline(ucgen.tiny(g["seed"]))
    r = pdhg.solve(S, tol=1e-4, max_iter=100_000, adaptive=True)
    assert r.status == "optimal"
    xr, _ = ops.postsolve(ps, S.Dc * r.x)
    assert abs(float(raw.c @ xr) - g["objective"]) / abs(g["objective"]) <= 1e-4


def test_adaptive_steps_never_collapse():
    # |dy^T A dx| <= ||A||_2 ||dx|| ||dy|| <= ||A||_2 (omega ||dx||^2 + ||dy||^2 / omega) / 2,
    # so eta_bar >= 1 / ||A||_2 at every attempt, and the trial step stays at or
    # above min(eta_0, (1 - 2^-0.3) / ||A||_2)
    raw, ps, S = _pipeline(_small(1))
    norm = float(np.linalg.norm(S.A.toarray(), 2))
    att = []
    pdhg.solve(S, tol=0.0, max_iter=3000, adaptive=True, attempts=att)
    floor = min(S.eta, (1.0 - 2.0 ** -0.3) / norm)
    for acc, eta, eta_bar in att:
        assert eta_bar >= (1.0 - 1e-12) / norm
        assert eta >= floor * (1.0 - 1e-12)


def test_adaptive_acceptance_is_the_pdhg_metric_test():
    # The rule bounds |dy^T A dx|, so a step is accepted exactly when dz^T M dz >= 0
    # for dz = (dx, dy) and for (dx, -dy), M = [[omega/eta I, -A^T], [-A, 1/(eta omega) I]]
    # being the PDHG preconditioner of the trial step: the quadratic forms are
    # built here from the block matrix, not from eta_bar.
    raw, ps, S = _pipeline(_small(2))
    st = pdhg.initial_state(S)
    AT = S.A.T.tocsr()
    m, n = S.A.shape
    seen = {True: 0, False: 0}
    for _ in range(1500):
        x0, y0, eta, om = st.x.copy(), st.y.copy(), st.eta_try, st.omega
        # the trial point, recomputed independently of the attempt
        xt = np.clip(x0 - (eta / om) * (S.c - AT @ y0), S.l, S.u)
        yt = y0 + (eta * om) * (S.q - S.A @ (2 * xt - x0))
        yt[S.m_eq:] = np.maximum(yt[S.m_eq:], 0.0)
        dz = np.concatenate([xt - x0, yt - y0])
        dzr = np.concatenate([xt - x0, y0 - yt])
        M = sp.bmat([[sp.identity(n) * (om / eta), -AT], [-S.A, sp.identity(m) / (eta * om)]]).tocsr()
        q = min(float(dz @ (M @ dz)), float(dzr @ (M @ dzr)))
        scale = float(dz @ dz) / eta * max(om, 1.0 / om)
        acc, _, _ = pdhg.adaptive_attempt(S, st, AT)
        if abs(q) > 1e-9 * scale:
            assert acc == (q >= 0.0), (q, acc)
            seen[acc] += 1
        if acc:
            np.testing.assert_array_equal(st.x, xt)
    assert seen[True] > 0 and seen[False] > 0


def test_adaptive_average_is_step_weighted():
    raw, ps, S = _pipeline(_small(0))
    st = pdhg.initial_state(S)
    AT = S.A.T.tocsr()
    xs, ws = np.zeros_like(st.x), 0.0
    for _ in range(1500):
        acc, eta, _ = pdhg.adaptive_attempt(S, st, AT)
        if acc:
            xs = xs + eta * st.x
            ws += eta
    assert st.w_sum == pytest.approx(ws, rel=1e-13)
    np.testing.assert_allclose(st.x_sum / st.w_sum, xs / ws, rtol=1e-12, atol=1e-15)
    assert st.accepted < 1500 and st.k == 1500


def test_adaptive_exact_sums_move_only_rounding():
    # correctly rounded sums in the step bound change the first attempts' iterates
    # only at rounding level (the sensitivity the device parity tests measure)
    raw, ps, S = _pipeline(_small(0))
    a = pdhg.solve(S, tol=0.0, max_iter=64, adaptive=True)
    b = pdhg.solve(S, tol=0.0, max_iter=64, adaptive=True, exact_sums=True)
    assert np.max(np.abs(a.x - b.x)) <= 1e-11 * np.max(np.abs(a.x))
    assert np.max(np.abs(a.y - b.y)) <= 1e-11 * np.max(np.abs(a.y))


# ---------------------------------------------------------------------------
# absolute primal infeasibility (the reported 1e-5 figure)
# ---------------------------------------------------------------------------
def _abs_violation_by_loops(lp, x):
    """max over rows and bounds of the violation, one element at a time."""
    A = lp.A.tocsr()
    worst = 0.0
    for i in range(A.shape[0]):
        act = 0.0
        for k in range(A.indptr[i], A.indptr[i + 1]):
            act += A.data[k] * x[A.indices[k]]
        r = act - lp.q[i]
        v = abs(r) if i < lp.m_eq else max(-r, 0.0)
        worst = max(worst, v)
    for j in range(A.shape[1]):
        worst = max(worst, lp.l[j] - x[j], x[j] - lp.u[j])
    return worst


@pytest.mark.parametrize("seed", range(3))
def test_abs_primal_inf_matches_loops_and_vanishes_at_the_optimum(seed):
    P = ucgen.micro(seed, B=6, L=8, G=3, T=4)
    raw = olp.build_lp(P)
    ref = simplex.solve_lp(raw)
    scale = 1.0 + float(np.max(np.abs(raw.q)))
    # a basic optimal point is feasible to the simplex's tolerance
    assert kkt.abs_primal_inf(raw, ref.x) <= 1e-8 * scale
    assert _abs_violation_by_loops(raw, ref.x) <= 1e-8 * scale
    # random points, inside and outside the bounds
    rng = np.random.default_rng(seed)
    lo = np.where(np.isfinite(raw.l), raw.l, -50.0)
    hi = np.where(np.isfinite(raw.u), raw.u, 50.0)
    for _ in range(5):
        x = rng.uniform(lo - 10.0, hi + 10.0)
        got = kkt.abs_primal_inf(raw, x)
        want = _abs_violation_by_loops(raw, x)
        assert got == pytest.approx(want, rel=1e-12, abs=1e-12)
        assert got > 0.0
