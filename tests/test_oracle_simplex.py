"""Pins for O2 (dense bounded simplex) against brute force and closed forms."""
import numpy as np
import pytest

import ucgen
from oracle import brute, closed, kkt, lp as olp, simplex


def _random_lp(rng, n, m_eq, m_in):
    m = m_eq + m_in
    A = rng.uniform(-2, 2, size=(m, n))
    A[np.abs(A) < 0.3] = 0.0
    x0 = rng.uniform(0.2, 0.8, size=n)        # strictly feasible point
    q = A @ x0
    q[m_eq:] -= rng.uniform(0.0, 0.5, size=m_in)
    c = rng.uniform(-1, 1, size=n)
    l = np.zeros(n)
    u = np.ones(n)
    if n > 2:                                  # one half-bounded column, bounded
        if c[0] > 0:                           # on the side its cost pushes to
            l[0], u[0] = -1.0, np.inf
        else:
            l[0], u[0] = -np.inf, 2.0
    return A, q, c, l, u


@pytest.mark.parametrize("seed", range(12))
def test_simplex_matches_vertex_enumeration(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 6))
    m_eq = int(rng.integers(0, 2))
    m_in = int(rng.integers(1, 4))
    A, q, c, l, u = _random_lp(rng, n, m_eq, m_in)
    best, _ = brute.vertex_enum(A, q, c, l, u, m_eq)
    r = simplex.solve(A, q, c, l, u, m_eq)
    assert r.status == "optimal"
    assert abs(r.obj - best) <= 1e-9 * max(1.0, abs(best))


@pytest.mark.parametrize("seed", range(3))
def test_simplex_micro_uc_matches_vertex_enumeration(seed):
    P = ucgen.micro(seed, B=2, L=1, G=1, T=1)
    raw = olp.build_lp(P)
    best, _ = brute.vertex_enum(raw.A, raw.q, raw.c, raw.l, raw.u, raw.m_eq)
    r = simplex.solve_lp(raw)
    assert r.status == "optimal"
    assert abs(r.obj - best) <= 1e-9 * max(1.0, abs(best))


def _one_bus(pmax, c, cnl, csu, d, voll=10_000.0, pmin_frac=0.3):
    G = len(pmax)
    pmax = np.asarray(pmax, float)
    return ucgen.UCProblem(
        B=1, L=0, G=G, T=1, ref_bus=0,
        line_from=np.zeros(0, np.int32), line_to=np.zeros(0, np.int32),
        x_pu=np.zeros(0), fmax=np.zeros(0), gen_bus=np.zeros(G, np.int32),
        pmax=pmax, pmin=pmin_frac * pmax, ramp=0.5 * pmax,
        c_lin=np.asarray(c, float), c_nl=np.asarray(cnl, float), c_su=np.asarray(csu, float),
        u0=np.zeros(G), load=np.array([[float(d)]]), voll=voll)


@pytest.mark.parametrize("d", [37.0, 200.0, 333.0, 610.0])
def test_simplex_one_bus_merit_order(d):
    pmax, c, cnl, csu = [100, 200, 150, 120], [20, 35, 12, 50], [300, 150, 400, 200], [1000, 500, 2000, 800]
    P = _one_bus(pmax, c, cnl, csu, d)
    raw = olp.build_lp(P)
    r = simplex.solve_lp(raw)
    assert r.status == "optimal"
    obj, p, shed, lmp = closed.merit_order(P.pmax, P.c_lin, P.c_nl, P.c_su, d, P.voll)
    assert abs(r.obj - obj) <= 1e-9 * obj
    sol = olp.split_solution(P, raw, r.x, r.y)
    np.testing.assert_allclose(sol["p"][0], p, atol=1e-7)
    assert abs(sol["shed"][0, 0] - shed) <= 1e-7
    assert abs(sol["lmp"][0, 0] - lmp) <= 1e-7 * max(1.0, lmp)


def test_simplex_two_bus_congestion():
    P = ucgen.UCProblem(
        B=2, L=1, G=2, T=1, ref_bus=0,
        line_from=np.array([0], np.int32), line_to=np.array([1], np.int32),
        x_pu=np.array([0.1]), fmax=np.array([80.0]), gen_bus=np.array([0, 1], np.int32),
        pmax=np.array([300.0, 300.0]), pmin=np.array([0.0, 0.0]), ramp=np.array([150.0, 150.0]),
        c_lin=np.array([10.0, 50.0]), c_nl=np.array([0.0, 0.0]), c_su=np.array([0.0, 0.0]),
        u0=np.zeros(2), load=np.array([[0.0, 200.0]]), voll=10_000.0)
    raw = olp.build_lp(P)
    r = simplex.solve_lp(raw)
    assert r.status == "optimal"
    obj, flow, lmp0, lmp1 = closed.two_bus(10.0, 300.0, 50.0, 300.0, 200.0, 80.0)
    assert abs(r.obj - obj) <= 1e-9 * obj
    sol = olp.split_solution(P, raw, r.x, r.y)
    assert abs(sol["f"][0, 0] - flow) <= 1e-7
    np.testing.assert_allclose(sol["lmp"][0], [lmp0, lmp1], rtol=1e-9)
    # the line limit's shadow price (reduced cost of f at its upper bound) is the LMP spread
    lam = raw.c - raw.A.T @ r.y
    jf = int(np.flatnonzero(raw.col_kind == olp.COL_F)[0])
    assert abs(-lam[jf] - (lmp1 - lmp0)) <= 1e-7


@pytest.mark.parametrize("seed", range(3))
def test_simplex_strong_duality_and_kkt(seed):
    P = ucgen.micro(seed, B=6, L=8, G=3, T=4)
    raw = olp.build_lp(P)
    r = simplex.solve_lp(raw)
    assert r.status == "optimal"
    assert max(kkt.relative_kkt(raw, r.x, r.y)) <= 1e-9


def test_simplex_infeasible_and_unbounded():
    A = np.array([[1.0, 1.0]])
    r = simplex.solve(A, np.array([5.0]), np.array([1.0, 1.0]), np.zeros(2), np.ones(2), 1)
    assert r.status == "infeasible"
    r = simplex.solve(A, np.array([1.0]), np.array([-1.0, 0.0]), np.array([0.0, -np.inf]),
                      np.array([np.inf, np.inf]), 1)
    assert r.status == "unbounded"


@pytest.mark.parametrize("seed", range(4))
def test_simplex_agrees_with_highs(seed):
    from scipy.optimize import linprog
    P = ucgen.micro(seed, B=8, L=10, G=3, T=6)
    raw = olp.build_lp(P)
    r = simplex.solve_lp(raw)
    bounds = list(zip(np.where(np.isfinite(raw.l), raw.l, None), np.where(np.isfinite(raw.u), raw.u, None)))
    h = linprog(raw.c, A_ub=-raw.A[raw.m_eq:], b_ub=-raw.q[raw.m_eq:], A_eq=raw.A[:raw.m_eq],
                b_eq=raw.q[:raw.m_eq], bounds=bounds, method="highs")
    assert h.status == 0
    assert abs(r.obj - h.fun) <= 1e-8 * abs(h.fun)
