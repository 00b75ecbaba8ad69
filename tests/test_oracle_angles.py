"""Pins for the oracle's angle elimination (oracle/presolve.py eliminate_angles,
restore_angles): the free bus angles substituted out along a breadth-first
spanning tree, each non-tree line's flow row rewritten as Kirchhoff's voltage
law on its fundamental cycle.

* a 3-bus triangle whose one substituted row is derived by hand;
* any angle vector, with the flows its flow-definition rows imply, satisfies
  every substituted row, and restore_angles gives the angles back (the rows
  are implied by the flow definitions, and the tree recovers the angles);
* the angle-free LP has the raw LP's optimum (the golden simplex objective);
* the postsolved simplex optimum is primal and dual optimal on the raw LP
  (the angles' reduced costs vanish with the tree rows' recovered duals).

The last test plants plausible mistakes into a copy of eliminate_angles and
checks that one of the first two pins fails on it."""
import inspect
import textwrap

import numpy as np
import pytest

import ucgen
from oracle import kkt, lp as olp, presolve as ops


def _triangle():
    # buses 0 (reference), 1, 2; lines l0: 0->1 (x 0.1), l1: 1->2 (x 0.2), l2: 0->2 (x 0.5)
    P = ucgen.micro(0, B=3, L=3, G=1, T=1)
    P.ref_bus = 0
    P.line_from = np.array([0, 1, 0], np.int32)
    P.line_to = np.array([1, 2, 2], np.int32)
    P.x_pu = np.array([0.1, 0.2, 0.5])
    P.fmax = np.array([100.0, 100.0, 100.0])
    return P


def _check_triangle(elim):
    raw = olp.build_lp(_triangle())
    E = elim(raw)
    # breadth-first from bus 0 over its lines in row order: l0 reaches bus 1 and
    # l2 bus 2, so l1 is the one non-tree line.  theta_1 - theta_2 =
    # (theta_0 - theta_2) - (theta_0 - theta_1) = x2 f2 - x0 f0, so its row
    # f1 - (theta_1 - theta_2) / x1 = 0 becomes f1 + (x0/x1) f0 - (x2/x1) f2 = 0:
    # coefficients 1, 0.5, -2.5 (stored 1/x: 10, 5, 2)
    th = np.flatnonzero(raw.col_kind == olp.COL_TH)
    assert not np.isin(th, E.col_keep).any()
    flow = np.flatnonzero(raw.row_kind == olp.ROW_FLOW)
    kept_flow = [i for i in flow if i in set(E.row_keep.tolist())]
    assert [int(raw.row_idx[i]) for i in kept_flow] == [1]
    r = int(np.flatnonzero(E.row_keep == kept_flow[0])[0])
    A = E.lp.A.tocsr()
    fcol = {int(raw.col_idx[j]): k for k, j in enumerate(E.col_keep) if raw.col_kind[j] == olp.COL_F}
    row = {int(A.indices[k]): float(A.data[k]) for k in range(A.indptr[r], A.indptr[r + 1])}
    assert row == pytest.approx({fcol[1]: 1.0, fcol[0]: 0.5, fcol[2]: -2.5}, rel=1e-15)
    assert E.lp.q[r] == 0.0
    assert E.lp.m_eq == raw.m_eq - 2


def _check_kvl_holds(elim):
    P = ucgen.tiny(1)     # two of its 12 non-tree lines' tree paths share edges below the root
    raw = olp.build_lp(P)
    E = elim(raw)
    rng = np.random.default_rng(5)
    x = rng.uniform(-1.0, 1.0, raw.n)
    th = raw.col_kind == olp.COL_TH
    x[th & (raw.l == 0.0) & (raw.u == 0.0)] = 0.0
    A = raw.A.tocsr()
    for i in np.flatnonzero(raw.row_kind == olp.ROW_FLOW):   # the flows the angles imply
        ents = range(A.indptr[i], A.indptr[i + 1])
        fc = [A.indices[k] for k in ents if raw.col_kind[A.indices[k]] == olp.COL_F][0]
        x[fc] = -sum(A.data[k] * x[A.indices[k]] for k in ents if A.indices[k] != fc)
    xk = x[E.col_keep]
    res = E.lp.A @ xk
    flow_rows = E.lp.row_kind == olp.ROW_FLOW
    assert np.max(np.abs(res[flow_rows])) <= 1e-12 * np.max(np.abs(xk))
    # the other rows are the raw rows without angle entries
    np.testing.assert_array_equal(res[~flow_rows], (A @ x)[E.row_keep[~flow_rows]])
    xr, _ = ops.restore_angles(E, raw, xk)
    np.testing.assert_allclose(xr, x, rtol=0, atol=1e-12)


PINS = [_check_triangle, _check_kvl_holds]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__[7:])
def test_angle_elimination_pins(pin):
    pin(ops.eliminate_angles)


@pytest.mark.parametrize("seed", [0, 2])
def test_angle_free_lp_has_the_raw_optimum(seed):
    from gpu_common import golden_tiny
    from oracle import simplex
    raw = olp.build_lp(ucgen.tiny(seed))
    ps = ops.presolve(raw, angles=True)
    r = simplex.solve_lp(ps.lp)
    opt = golden_tiny()["objective_by_seed"][str(seed)]
    assert (r.obj + ps.lp.obj_const) == pytest.approx(opt, rel=1e-9)
    xr, yr = ops.postsolve(ps, r.x, r.y)
    assert float(raw.c @ xr) + raw.obj_const == pytest.approx(opt, rel=1e-9)
    # every raw row holds, tree and non-tree flow rows included, and the pair
    # is KKT-optimal on the raw LP (angle columns: zero reduced cost)
    assert kkt.abs_primal_inf(raw, xr) <= 1e-8 * max(1.0, float(np.max(np.abs(raw.q))))
    assert max(kkt.relative_kkt(raw, xr, yr)) <= 1e-8
    lam = raw.c - raw.A.T @ yr
    th = raw.col_kind == olp.COL_TH
    assert np.max(np.abs(lam[th])) <= 1e-8 * max(1.0, float(np.max(np.abs(yr))))


MUTANTS = {
    "child end taken the wrong way": [("1.0 if edges[e][2] == v else -1.0", "1.0 if edges[e][3] == v else -1.0")],
    "b's path with a's sign": [("row[edges[g][1]] = sg * inv / edges[g][4]", "row[edges[g][1]] = -sg * inv / edges[g][4]")],
    "ratio of reactances inverted": [("-sg * inv / edges[g][4]", "-sg * edges[g][4] / inv"),
                                     ("row[edges[g][1]] = sg * inv / edges[g][4]", "row[edges[g][1]] = sg * edges[g][4] / inv")],
    "common part of the paths kept": [("while pa and pb and pa[-1] == pb[-1]:", "while False:")],
    "line's own flow dropped": [("row = {fc: 1.0}", "row = {}")],
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_each_planted_mistake_fails_a_pin(name):
    src = textwrap.dedent(inspect.getsource(ops.eliminate_angles))
    for old, new in MUTANTS[name]:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    ns = dict(vars(ops))
    exec(compile(src, "<mutant>", "exec"), ns)
    bad = ns["eliminate_angles"]
    failed = []
    for pin in PINS:
        try:
            pin(bad)
        except (AssertionError, KeyError, ValueError):
            failed.append(pin.__name__)
    assert failed, f"no pin caught the planted mistake: {name}"


def test_parallel_lines_form_a_two_entry_cycle():
    # two lines between the same buses form a 2-entry cycle: the second line's
    # row becomes f_1 - (x_0 / x_1) f_0 = 0
    P = _triangle()
    P.line_from = np.array([0, 0, 1], np.int32)
    P.line_to = np.array([1, 1, 2], np.int32)
    P.x_pu = np.array([0.1, 0.4, 0.5])
    raw = olp.build_lp(P)
    E = ops.eliminate_angles(raw)
    fcol = {int(raw.col_idx[j]): k for k, j in enumerate(E.col_keep) if raw.col_kind[j] == olp.COL_F}
    kept = [i for i in np.flatnonzero(raw.row_kind == olp.ROW_FLOW) if i in set(E.row_keep.tolist())]
    assert [int(raw.row_idx[i]) for i in kept] == [1]
    r = int(np.flatnonzero(E.row_keep == kept[0])[0])
    A = E.lp.A.tocsr()
    row = {int(A.indices[k]): float(A.data[k]) for k in range(A.indptr[r], A.indptr[r + 1])}
    # theta_0 - theta_1 = x0 f0 (tree line 0 from the reference bus), so
    # f1 - (theta_0 - theta_1) / x1 = f1 - (x0 / x1) f0 = f1 - 0.25 f0
    assert row == pytest.approx({fcol[1]: 1.0, fcol[0]: -0.25}, rel=1e-15)
    _check_kvl_on(raw, E)


def _check_kvl_on(raw, E):
    rng = np.random.default_rng(3)
    x = rng.uniform(-1.0, 1.0, raw.n)
    th = raw.col_kind == olp.COL_TH
    x[th & (raw.l == 0.0) & (raw.u == 0.0)] = 0.0
    A = raw.A.tocsr()
    for i in np.flatnonzero(raw.row_kind == olp.ROW_FLOW):
        ents = range(A.indptr[i], A.indptr[i + 1])
        fc = [A.indices[k] for k in ents if raw.col_kind[A.indices[k]] == olp.COL_F][0]
        x[fc] = -sum(A.data[k] * x[A.indices[k]] for k in ents if A.indices[k] != fc)
    xk = x[E.col_keep]
    res = E.lp.A @ xk
    assert np.max(np.abs(res[E.lp.row_kind == olp.ROW_FLOW])) <= 1e-12 * np.max(np.abs(xk))
    xr, _ = ops.restore_angles(E, raw, xk)
    np.testing.assert_allclose(xr, x, rtol=0, atol=1e-12)
