"""Postsolve on the GPU path: the duals uc_get_raw_solution recovers (removed
singleton rows included) and the LMPs uc_get_solution reports, after a device
solve through the C ABI.

* One bus, one period: the LMP is the effective cost of the marginal unit
  (merit-order closed form) or VOLL when load is shed.
* Two buses, one congested line: each bus is priced by its own unit and the
  line limit's shadow price (minus the reduced cost of f at its upper bound)
  is the LMP difference.
* The 30-bus LP with a zero-limit line at the reference bus: presolve turns
  that line's flow row into singleton rows that fix bus angles, and postsolve
  must give each of them the dual that zeroes the free angle's reduced cost.
  The full raw dual must equal the oracle's postsolve of the same presolved
  point, the postsolved pair must meet the KKT tolerance on the RAW LP (where
  the recovered duals matter: without them the dual residual is about 6), and
  the LMP array must be the balance rows' duals.

The closed forms hold at the LP optimum; the solves here run to relative KKT
1e-8, at which the oracle PDHG's LMPs sit within 1.1e-8 of them (measured on
the same instances), so 1e-6 leaves a wide margin.  At the paper's 1e-4 the
LMPs are within 2e-4 relative (also checked).
"""
import numpy as np
import pytest

import ucgen
from gpu_common import ITERATE_RTOL, KKT_TOL
from oracle import closed, kkt, lp as olp, presolve as ops

pytestmark = pytest.mark.gpu

LMP_RTOL_TIGHT = 1e-6     # solves to relative KKT 1e-8
LMP_RTOL_PAPER = 1e-3     # solves to relative KKT 1e-4


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_03627_gb300 as pkg
    pkg.build()
    from paper_2607_03627_gb300 import binding
    return binding


def _one_bus(pmax, c, cnl, csu, d, voll=10_000.0):
    G = len(pmax)
    pmax = np.asarray(pmax, float)
    return ucgen.UCProblem(
        B=1, L=0, G=G, T=1, ref_bus=0,
        line_from=np.zeros(0, np.int32), line_to=np.zeros(0, np.int32),
        x_pu=np.zeros(0), fmax=np.zeros(0), gen_bus=np.zeros(G, np.int32),
        pmax=pmax, pmin=0.3 * pmax, ramp=0.5 * pmax,
        c_lin=np.asarray(c, float), c_nl=np.asarray(cnl, float), c_su=np.asarray(csu, float),
        u0=np.zeros(G), load=np.array([[float(d)]]), voll=voll)


@pytest.mark.parametrize("tol,rtol", [(1e-8, LMP_RTOL_TIGHT), (KKT_TOL, LMP_RTOL_PAPER)])
@pytest.mark.parametrize("d", [37.0, 200.0, 333.0, 610.0])
def test_one_bus_lmp_is_the_marginal_cost(B, d, tol, rtol):
    pmax, c, cnl, csu = [100, 200, 150, 120], [20, 35, 12, 50], [300, 150, 400, 200], [1000, 500, 2000, 800]
    P = _one_bus(pmax, c, cnl, csu, d)
    obj, p, shed, lmp = closed.merit_order(P.pmax, P.c_lin, P.c_nl, P.c_su, d, P.voll)
    res, rc = B.uc_solve(B.uc_presolve(B.uc_build_lp(P)), tol=tol)
    assert rc == B.UC_OK
    sol = B.uc_get_solution(res, P.T, P.B, P.L, P.G)
    assert sol["lmp"][0, 0] == pytest.approx(lmp, rel=rtol)
    assert sol["stats"]["objective"] == pytest.approx(obj, rel=max(tol, 1e-9))


@pytest.mark.parametrize("tol,rtol", [(1e-8, LMP_RTOL_TIGHT), (KKT_TOL, LMP_RTOL_PAPER)])
def test_two_bus_lmps_and_line_shadow_price(B, tol, rtol):
    P = ucgen.UCProblem(
        B=2, L=1, G=2, T=1, ref_bus=0,
        line_from=np.array([0], np.int32), line_to=np.array([1], np.int32),
        x_pu=np.array([0.1]), fmax=np.array([80.0]), gen_bus=np.array([0, 1], np.int32),
        pmax=np.array([300.0, 300.0]), pmin=np.array([0.0, 0.0]), ramp=np.array([150.0, 150.0]),
        c_lin=np.array([10.0, 50.0]), c_nl=np.array([0.0, 0.0]), c_su=np.array([0.0, 0.0]),
        u0=np.zeros(2), load=np.array([[0.0, 200.0]]), voll=10_000.0)
    obj, flow, lmp0, lmp1 = closed.two_bus(10.0, 300.0, 50.0, 300.0, 200.0, 80.0)
    raw = olp.build_lp(P)
    res, rc = B.uc_solve(B.uc_presolve(B.uc_build_lp(P)), tol=tol)
    assert rc == B.UC_OK
    sol = B.uc_get_solution(res, P.T, P.B, P.L, P.G)
    np.testing.assert_allclose(sol["lmp"][0], [lmp0, lmp1], rtol=rtol)
    assert sol["f"][0, 0] == pytest.approx(flow, rel=rtol)
    xr, yr = B.uc_get_raw_solution(res, raw.n, raw.m)
    lam = raw.c - raw.A.T @ yr
    jf = int(np.flatnonzero(raw.col_kind == olp.COL_F)[0])
    assert -lam[jf] == pytest.approx(lmp1 - lmp0, rel=rtol)


def _zero_limit_line_at_ref():
    P = ucgen.tiny(0)
    l = int(np.flatnonzero((P.line_from == P.ref_bus) | (P.line_to == P.ref_bus))[0])
    P.fmax[l] = 0.0
    return P


def test_recovered_duals_and_lmps_match_oracle_postsolve(B):
    P = _zero_limit_line_at_ref()
    raw = olp.build_lp(P)
    ps_o = ops.presolve(raw)
    S = ops.scale(ps_o.lp)
    tightened = [r for r in ps_o.removed_rows if r[4]]
    assert len(tightened) >= P.T                 # one angle-fixing row per period at least
    ps = B.uc_presolve(B.uc_build_lp(P))
    res, rc = B.uc_solve(ps, tol=KKT_TOL)
    assert rc == B.UC_OK
    n, m, _, _ = B.uc_presolved_dims(ps)
    assert (n, m) == (ps_o.lp.n, ps_o.lp.m)
    xs, ys = B.uc_get_iterate(res, 2, n, m)     # the returned point, scaled presolved LP
    xr_o, yr_o = ops.postsolve(ps_o, S.Dc * xs, S.Dr * ys)
    xr, yr = B.uc_get_raw_solution(res, raw.n, raw.m)
    scale_x = np.max(np.abs(xr_o))
    scale_y = np.max(np.abs(yr_o))
    assert np.max(np.abs(xr - xr_o)) <= ITERATE_RTOL * scale_x
    assert np.max(np.abs(yr - yr_o)) <= ITERATE_RTOL * scale_y
    rows = np.array([r[0] for r in tightened])
    assert np.all(np.abs(yr[rows]) > 1.0)        # the recovered duals are not trivially zero
    # the postsolved pair is KKT-optimal on the raw LP only with those duals
    assert max(kkt.relative_kkt(raw, xr, yr)) <= KKT_TOL * (1 + 1e-6)
    y0 = yr.copy()
    y0[rows] = 0.0
    assert kkt.relative_kkt(raw, xr, y0)[1] > 1.0
    # the LMP array is the balance rows' duals, period-major
    sol = B.uc_get_solution(res, P.T, P.B, P.L, P.G)
    ref = olp.split_solution(P, raw, xr_o, yr_o)["lmp"]
    assert np.max(np.abs(sol["lmp"] - ref)) <= ITERATE_RTOL * np.max(np.abs(ref))
