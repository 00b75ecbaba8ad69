"""Pins of the oracle's infeasibility detection (Halpern PDHG, every 4th
evaluation, Farkas direction from the last step's dual residual).

* On strict-model instances (no load shedding) whose demand exceeds the
  generation capacity, the simplex reports infeasible and the PDHG stops with
  "infeasible".
* The direction it returns is checked against the primal side, with no use of
  the projection formula the detection uses: y with y_I >= 0 implies
  y.(A x - q) >= 0 for every feasible x, so when the largest value of y.A x
  over a box holding every feasible x is below y.q, no x can be feasible.
  The free bus angles get the box |theta| <= sum over lines of x_l F_l, which
  every feasible point meets (theta_ref = 0 and each line fixes the angle
  difference to x_l f_l with |f_l| <= F_l).
* A hand-built one-bus LP: the direction is a positive multiple of the
  balance rows' duals, as Farkas' lemma predicts for demand above capacity.
* Feasible instances never stop as infeasible.
"""
import numpy as np
import pytest

import ucgen
from oracle import kkt, lp as olp, pdhg, presolve as ops, simplex


def _strict_pipeline(P):
    raw = olp.build_lp(P)
    ps = ops.presolve(raw)
    S = ops.scale(ps.lp)
    return raw, ps, S


def _box_max(g, l, u):
    """max of g.x over l <= x <= u (inf when unbounded in a direction g pushes)."""
    tot = 0.0
    for gj, lj, uj in zip(g, l, u):
        if gj > 0:
            if not np.isfinite(uj):
                return np.inf
            tot += gj * uj
        elif gj < 0:
            if not np.isfinite(lj):
                return np.inf
            tot += gj * lj
    return tot


INFEASIBLE_CASES = [
    dict(seed=3, B=12, L=16, G=3, T=4, lo=1.05, hi=1.2),
    dict(seed=5, B=8, L=10, G=2, T=3, lo=1.1, hi=1.3),
    dict(seed=8, B=20, L=26, G=4, T=6, lo=1.02, hi=1.1),
]


@pytest.mark.parametrize("case", INFEASIBLE_CASES)
def test_detects_infeasible_strict_instances(case):
    c = dict(case)
    P = ucgen.make_problem(c.pop("seed"), voll=0.0, **c)
    raw, ps, S = _strict_pipeline(P)
    assert simplex.solve_lp(ps.lp).status == "infeasible"
    res = pdhg.solve_halpern(S, tol=1e-4, max_iter=100_000)
    assert res.status == "infeasible"
    assert res.iters % (pdhg.N_EVAL * pdhg.INFEAS_EVERY) == 0
    # the direction in the unscaled presolved LP proves infeasibility from the primal side
    lp = ps.lp
    y = S.Dr * res.y
    y_clean = y.copy()   # the proof below needs y_I >= 0 exactly
    y_clean[lp.m_eq:] = np.maximum(y_clean[lp.m_eq:], 0.0)
    R = float(np.sum(P.x_pu * P.fmax))
    l_box = np.where(np.isfinite(lp.l), lp.l, -R)
    u_box = np.where(np.isfinite(lp.u), lp.u, R)
    assert _box_max(lp.A.T @ y_clean, l_box, u_box) < float(lp.q @ y_clean)


def test_one_bus_direction_is_the_balance_dual():
    # one bus, two periods, two units (Pmax 50 and 30), demand 100 in both
    # periods: columns p1, p2 in [0, Pmax] with rows p1 + p2 = 100 per period
    import scipy.sparse as sp

    class LP:
        pass
    lp = LP()
    lp.A = sp.csr_matrix(np.array([[1.0, 1.0, 0.0, 0.0], [0.0, 0.0, 1.0, 1.0]]))
    lp.q = np.array([100.0, 100.0])
    lp.c = np.array([10.0, 20.0, 10.0, 20.0])
    lp.l = np.zeros(4)
    lp.u = np.array([50.0, 30.0, 50.0, 30.0])
    lp.m_eq = 2
    lp.n, lp.m = 4, 2
    lp.obj_const = 0.0
    S = ops.scale(lp)
    res = pdhg.solve_halpern(S, tol=1e-4, max_iter=20_000)
    assert res.status == "infeasible"
    y = S.Dr * res.y
    # Farkas: y > 0 on both balance rows (more power is needed than exists);
    # its objective is (100 - 80) (y_1 + y_2) > 0
    assert np.all(y > 0)
    obj, viol = kkt.farkas_ray(lp, y)
    assert obj == pytest.approx(20.0 * (y[0] + y[1]), rel=1e-6)
    assert viol <= 1e-8 * obj


def test_farkas_test_rejects_feasible_directions():
    # on a feasible LP no direction can pass: random directions all fail
    P = ucgen.tiny(0)
    raw, ps, S = _strict_pipeline(P)
    rng = np.random.default_rng(0)
    for _ in range(50):
        y = rng.standard_normal(ps.lp.m)
        y[ps.lp.m_eq:] = np.abs(y[ps.lp.m_eq:])
        assert not kkt.is_infeasibility_certificate(ps.lp, y)


@pytest.mark.parametrize("seed", range(3))
def test_feasible_instances_never_stop_as_infeasible(seed):
    P = ucgen.tiny(seed)
    _, _, S = _strict_pipeline(P)
    res = pdhg.solve_halpern(S, tol=1e-4)
    assert res.status == "optimal"
