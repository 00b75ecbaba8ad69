"""Pins for the oracle's primal feasibility polishing (pdhg.polish_primal): the
paper's PDHG settings pair the 1e-4 convergence tolerance with an absolute
feasibility tolerance of 1e-5 (Sec. II-D).  Polishing runs the Halpern PDHG on
the feasibility problem (objective 0) from a solve's primal point.

* After a 1e-4 solve of the 30-bus LPs, the polished point violates no row of
  the RAW LP by more than 1e-5 (the absolute-violation figure is pinned by
  element loops elsewhere) and its objective stays within 1e-4 of the
  simplex optimum.
* A start that is already feasible is a fixed point of the feasibility map:
  from the simplex optimum, polishing stops at its first evaluation without
  moving it.
* On one equality row over a box, from an infeasible start, it ends on the
  row (closed form of feasibility) inside the box.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

import ucgen
from oracle import kkt, lp as olp, pdhg, presolve as ops, simplex

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("seed", range(4))
def test_polish_meets_absolute_tolerance_and_keeps_the_objective(seed):
    with open(os.path.join(GOLDEN, "tiny_lp.json")) as f:
        opt = json.load(f)["objective_by_seed"][str(seed)]
    raw = olp.build_lp(ucgen.tiny(seed))
    ps = ops.presolve(raw)
    S = ops.scale(ps.lp)
    r = pdhg.solve_halpern(S, tol=1e-4)
    xr0, _ = ops.postsolve(ps, S.Dc * r.x)
    before = kkt.abs_primal_inf(raw, xr0)
    p = pdhg.polish_primal(S, r.x, 1e-5, omega0=r.omega)
    assert p.status == "optimal" and p.iters > 0
    xr, _ = ops.postsolve(ps, S.Dc * p.x)
    assert kkt.abs_primal_inf(raw, xr) <= 1e-5 < before
    assert abs(float(raw.c @ xr) - opt) / abs(opt) <= 1e-4


def test_polish_leaves_a_feasible_point_in_place():
    raw = olp.build_lp(ucgen.micro(1, B=6, L=8, G=3, T=4))
    ps = ops.presolve(raw)
    S = ops.scale(ps.lp)
    ref = simplex.solve_lp(ps.lp)
    assert ref.status == "optimal"
    xs = ref.x / S.Dc
    p = pdhg.polish_primal(S, xs, 1e-5)
    assert p.status == "optimal" and p.iters == pdhg.N_EVAL
    assert np.max(np.abs(p.x - xs)) <= 1e-9 * max(1.0, np.max(np.abs(xs)))


def test_polish_single_row_lands_on_the_row():
    lp = olp.LP(A=sp.csr_matrix(np.array([[1.0, 2.0, 1.0]])), q=np.array([2.0]), c=np.array([5.0, 1.0, 3.0]),
                l=np.zeros(3), u=np.ones(3), m_eq=1)
    S = ops.scale(lp)
    x0 = np.array([0.9, 0.9, 0.9]) / S.Dc                     # row value 3.6 != 2
    p = pdhg.polish_primal(S, x0, 1e-8, max_iter=100_000)
    x = S.Dc * p.x
    assert p.status == "optimal"
    assert abs(x[0] + 2 * x[1] + x[2] - 2.0) <= 1e-8
    assert np.all(x >= -1e-12) and np.all(x <= 1 + 1e-12)
