"""Pins for the oracle's vertex test (oracle.vertex.is_vertex), then the host
crossover (uc_crossover) judged by it.

The test itself: the corners of a box LP are vertices and its centre is not;
the simplex optimum of a micro UC LP (a basic solution by construction) is a
vertex; the midpoint of two different vertices is not; an infeasible point is
not.  The crossover: from the oracle PDHG's 1e-4 point on the presolved
30-bus LP (host only, through uc_result_from_point), uc_crossover must end at
a vertex of the presolved LP whose objective equals the simplex optimum within
1e-9, with a KKT residual of round-off size."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

import ucgen
from oracle import kkt, lp as olp, pdhg, presolve as ops, simplex, vertex

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _box():
    # x1 + x2 >= 0.5 over the unit box
    return olp.LP(A=sp.csr_matrix(np.array([[1.0, 1.0]])), q=np.array([0.5]), c=np.array([1.0, 1.0]),
                  l=np.zeros(2), u=np.ones(2), m_eq=0)


def test_vertex_test_on_a_box():
    lp = _box()
    assert vertex.is_vertex(lp, np.array([1.0, 1.0]))
    assert vertex.is_vertex(lp, np.array([0.5, 0.0]))          # on the row and a bound
    assert not vertex.is_vertex(lp, np.array([0.5, 0.5]))      # interior of the feasible set
    assert not vertex.is_vertex(lp, np.array([0.25, 0.25]))    # on the row only
    assert not vertex.is_vertex(lp, np.array([0.0, 0.0]))      # a corner that violates the row


def test_simplex_optimum_is_a_vertex_and_midpoints_are_not():
    raw = olp.build_lp(ucgen.micro(1, B=6, L=8, G=3, T=4))
    lp = ops.presolve(raw).lp
    r = simplex.solve_lp(lp)
    assert r.status == "optimal" and vertex.is_vertex(lp, r.x)
    # another vertex: the optimum for a different cost; their midpoint is no vertex
    lp2 = olp.LP(A=lp.A, q=lp.q, c=-lp.c + 1.0, l=lp.l, u=lp.u, m_eq=lp.m_eq)
    r2 = simplex.solve_lp(lp2)
    assert r2.status == "optimal" and vertex.is_vertex(lp, r2.x)
    assert np.max(np.abs(r.x - r2.x)) > 1e-6
    assert not vertex.is_vertex(lp, 0.5 * (r.x + r2.x))


@pytest.fixture(scope="module")
def B():
    import paper_2607_03627_gb300 as pkg
    pkg.build()
    from paper_2607_03627_gb300 import binding
    return binding


def test_crossover_from_the_oracle_pdhg_point_reaches_the_simplex_vertex(B):
    with open(os.path.join(GOLDEN, "tiny_lp.json")) as f:
        opt = json.load(f)["objective_by_seed"]["0"]
    P = ucgen.tiny(0)
    raw = olp.build_lp(P)
    ps_o = ops.presolve(raw)
    S = ops.scale(ps_o.lp)
    r = pdhg.solve_halpern(S, tol=1e-4)
    assert not vertex.is_vertex(ps_o.lp, S.Dc * r.x)           # PDHG ends off the vertices
    ps = B.uc_presolve(B.uc_build_lp(P))
    v, rc = B.uc_crossover(B.uc_result_from_point(ps, r.x, r.y))
    assert rc == B.UC_OK
    st = B.uc_get_stats(v)
    assert st["superbasic"] == 0
    xr, yr = B.uc_get_raw_solution(v, raw.n, raw.m)
    assert vertex.is_vertex(ps_o.lp, xr[ps_o.col_map])
    assert abs(float(raw.c @ xr) - opt) <= 1e-9 * abs(opt)
    assert max(kkt.relative_kkt(raw, xr, yr)) <= 1e-9


def test_crossover_rejects_results_without_a_point_and_big_lps(B):
    P = ucgen.paper_scale(0)
    ps = B.uc_presolve(B.uc_build_lp(P), power_max_iter=1)
    n, m, _, _ = B.uc_presolved_dims(ps)
    res = B.uc_result_from_point(ps, np.zeros(n), np.zeros(m))
    with pytest.raises(B.UCError, match="rows"):
        B.uc_crossover(res)


def test_host_simplex_arm_reaches_the_simplex_optimum(B):
    # the CPU arm of the concurrent solve, from the cold start, on a micro UC LP
    P = ucgen.micro(2, B=5, L=6, G=3, T=3)
    raw = olp.build_lp(P)
    ps_o = ops.presolve(raw)
    ref = simplex.solve_lp(raw)
    r, rc = B.uc_simplex_solve(B.uc_presolve(B.uc_build_lp(P)))
    assert rc == B.UC_OK and B.uc_get_stats(r)["superbasic"] == 0
    xr, yr = B.uc_get_raw_solution(r, raw.n, raw.m)
    assert abs(float(raw.c @ xr) - ref.obj) <= 1e-9 * abs(ref.obj)
    assert vertex.is_vertex(ps_o.lp, xr[ps_o.col_map])


def test_host_simplex_arm_stops_when_cancelled(B):
    import ctypes
    import threading
    import time
    ps = B.uc_presolve(B.uc_build_lp(ucgen.tiny(1)))
    flag = ctypes.c_int(0)
    timer = threading.Timer(0.2, lambda: setattr(flag, "value", 1))
    timer.start()
    t0 = time.perf_counter()
    with pytest.raises(B.UCError, match="cancelled"):
        B.uc_simplex_solve(ps, cancel=flag)
    assert time.perf_counter() - t0 < 5.0
