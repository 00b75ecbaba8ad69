"""GPU parity of the device PDHG (through the C ABI) against the CPU oracle."""
import ctypes

import numpy as np
import pytest

import ucgen
from gpu_common import (ITERATE_RTOL, KKT_TOL, OBJ_GAP_TOL, golden_tiny, oracle_kkt_of_raw,
                        oracle_pipeline, oracle_solve, oracle_trace, raw_objective, rel_inf)
from oracle import kkt, lp as olp, pdhg, simplex

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_03627_gb300 as pkg
    pkg.build()
    from paper_2607_03627_gb300 import binding
    return binding


def _device_iterates(B, ps, n, m, K, **kw):
    res, rc = B.uc_solve(ps, tol=0.0, max_iter=K, **kw)
    assert rc == B.UC_EITERLIMIT
    x, y = B.uc_get_iterate(res, 0, n, m)
    st = B.uc_get_stats(res)
    return x, y, st


KS = [1, 2, 3, 17, 63, 64, 65, 127, 128, 129, 191, 192, 193, 200]


VARIANTS = [("halpern", "kkt"), ("halpern", "fpr"), ("halpern", "fprp"), ("average", "kkt")]


@pytest.mark.parametrize("variant,metric", VARIANTS)
@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("which", ["tiny", "small_ragged"])
def test_per_iterate_parity_first_200(B, which, use_graph, variant, metric):
    if which == "tiny":
        P = ucgen.tiny(0)
    else:  # sizes far from the 256-row tiles, zero-Pmin units
        P = ucgen.make_problem(7, B=37, L=53, G=11, T=5, lo=0.5, hi=0.9, noise=0.05, zero_pmin_frac=0.2)
    raw, ps_o, S = oracle_pipeline(P)
    ref = oracle_trace(S, KS, variant=variant, metric=metric)
    ps = B.uc_presolve(B.uc_build_lp(P))
    n, m, _, _ = B.uc_presolved_dims(ps)
    for K in KS:
        x, y, st = _device_iterates(B, ps, n, m, K, use_graph=use_graph, algorithm=variant,
                                    restart_metric=metric)
        xo, yo, restarts, omega, xm, ym = ref[K]
        assert st["iters"] == K
        assert st["restarts"] == restarts, f"restart decision differs at K={K}"
        assert rel_inf(x, xo) <= ITERATE_RTOL, (K, rel_inf(x, xo))
        assert rel_inf(y, yo) <= ITERATE_RTOL, (K, rel_inf(y, yo))
        assert st["omega"] == pytest.approx(omega, rel=1e-9)
        if xm is not None:   # the PDHG map output the Halpern step came from
            res, _ = B.uc_solve(ps, tol=0.0, max_iter=K, use_graph=use_graph, algorithm=variant,
                                restart_metric=metric)
            xr, yr = B.uc_get_iterate(res, 2, n, m)
            assert rel_inf(xr, xm) <= ITERATE_RTOL and rel_inf(yr, ym) <= ITERATE_RTOL


@pytest.mark.parametrize("variant,metric", VARIANTS)
@pytest.mark.parametrize("seed", range(4))
def test_tiny_solve_meets_gates(B, seed, variant, metric):
    g = golden_tiny()
    P = ucgen.tiny(seed)
    raw, ps_o, S = oracle_pipeline(P)
    ps = B.uc_presolve(B.uc_build_lp(P))
    res, rc = B.uc_solve(ps, tol=KKT_TOL, algorithm=variant, restart_metric=metric)
    assert rc == B.UC_OK
    st = B.uc_get_stats(res)
    xr, yr = B.uc_get_raw_solution(res, raw.n, raw.m)
    assert max(oracle_kkt_of_raw(ps_o, xr, yr)) <= KKT_TOL * (1 + 1e-6)
    opt = g["objective_by_seed"][str(seed)]
    # PDLP iterate averaging (an option; no benchmark configuration uses it) stops
    # on the same relative KKT, whose gap part has the denominator 1 + |pobj| +
    # |dobj|, about 2 |obj|, so it bounds the objective error only by about 2e-4
    # of |obj| (more with the primal residual); on seed 3 the averaged point is
    # off by 2.3e-4, where the Halpern variant stays below 1e-6
    gap_tol = OBJ_GAP_TOL if variant == "halpern" else 3 * OBJ_GAP_TOL
    assert abs(raw_objective(raw, xr) - opt) / max(1.0, abs(opt)) <= gap_tol
    assert st["objective"] == pytest.approx(raw_objective(raw, xr), rel=1e-12)
    # the oracle PDHG takes the same path to the same stop
    r = oracle_solve(S, KKT_TOL, variant, metric)
    assert r.iters == st["iters"] and r.restarts == st["restarts"]
    # power balance of the returned dispatch, per period (satisfied to the tolerance)
    sol = B.uc_get_solution(res, P.T, P.B, P.L, P.G)
    bal = sol["p"].sum(axis=1) + sol["shed"].sum(axis=1) - P.load.sum(axis=1)
    assert np.max(np.abs(bal)) <= 1e-3 * P.load.sum(axis=1).max()


def test_fp32_values_meet_gates_and_report_error(B):
    g = golden_tiny()
    P = ucgen.tiny(0)
    raw, ps_o, S = oracle_pipeline(P)
    lp = B.uc_build_lp(P)
    r64, _ = B.uc_solve(B.uc_presolve(lp), tol=KKT_TOL)
    r32, rc = B.uc_solve(B.uc_presolve(lp, value_bits=32), tol=KKT_TOL)
    assert rc == B.UC_OK
    xr, yr = B.uc_get_raw_solution(r32, raw.n, raw.m)
    assert max(oracle_kkt_of_raw(ps_o, xr, yr)) <= 1.1 * KKT_TOL    # FP64 LP, FP32-stored matrix
    assert abs(raw_objective(raw, xr) - g["objective"]) / g["objective"] <= OBJ_GAP_TOL
    x64, _ = B.uc_get_raw_solution(r64, raw.n, raw.m)
    # error of the FP32-value path against the FP64 path at the same tolerance
    err = abs(raw_objective(raw, xr) - raw_objective(raw, x64)) / g["objective"]
    assert err <= 2 * OBJ_GAP_TOL


def test_batch_equals_single_solves(B):
    Ps = [ucgen.tiny(s) for s in range(3)] + [ucgen.micro(5, B=9, L=12, G=3, T=4)]
    pss = [B.uc_presolve(B.uc_build_lp(P)) for P in Ps]
    singles = [B.uc_solve(p, tol=KKT_TOL)[0] for p in pss]
    batch, rc = B.uc_solve_batch(pss, tol=KKT_TOL)
    assert rc == B.UC_OK
    for p, s, b in zip(pss, singles, batch):
        n, m, _, _ = B.uc_presolved_dims(p)
        xs, ys = B.uc_get_iterate(s, 2, n, m)
        xb, yb = B.uc_get_iterate(b, 2, n, m)
        np.testing.assert_array_equal(xb, xs)       # same arithmetic, same order
        np.testing.assert_array_equal(yb, ys)
        assert B.uc_get_stats(b)["iters"] == B.uc_get_stats(s)["iters"]


def test_edge_cases(B):
    P = ucgen.tiny(1)
    ps = B.uc_presolve(B.uc_build_lp(P))
    n, m, _, _ = B.uc_presolved_dims(ps)
    # max_iter 0: the starting point comes back unchanged
    res, rc = B.uc_solve(ps, tol=KKT_TOL, max_iter=0)
    assert rc == B.UC_EITERLIMIT
    x, y = B.uc_get_iterate(res, 0, n, m)
    d = B.uc_presolved_export(ps)
    np.testing.assert_array_equal(x, np.clip(0.0, d["l"], d["u"]))
    assert not y.any()
    # warm start from a converged point stops at the first evaluation
    res, rc = B.uc_solve(ps, tol=KKT_TOL)
    x, y = B.uc_get_iterate(res, 2, n, m)
    res2, rc2 = B.uc_solve(ps, tol=KKT_TOL * 1.5, warm_x=x, warm_y=y)
    assert rc2 == B.UC_OK and B.uc_get_stats(res2)["iters"] == 64
    # cancellation: a set flag stops the solve at the first replay boundary
    flag = ctypes.c_int(1)
    res3, rc3 = B.uc_solve(ps, tol=1e-12, cancel=flag)
    assert rc3 == B.UC_ECANCELLED
    assert B.uc_get_stats(res3)["iters"] <= 2 * 64
    # no units: only shed, flows and angles
    Q = ucgen.micro(3, B=4, L=5, G=1, T=2)
    Q.G = 0
    for f in ("gen_bus", "pmax", "pmin", "ramp", "c_lin", "c_nl", "c_su", "u0"):
        setattr(Q, f, getattr(Q, f)[:0])
    raw, ps_o, _ = oracle_pipeline(Q)
    psq = B.uc_presolve(B.uc_build_lp(Q))
    res, rc = B.uc_solve(psq, tol=KKT_TOL)
    assert rc == B.UC_OK
    xr, _ = B.uc_get_raw_solution(res, raw.n, raw.m)
    ref = simplex.solve_lp(raw)
    assert abs(raw_objective(raw, xr) - ref.obj) / ref.obj <= OBJ_GAP_TOL


@pytest.mark.parametrize("variant", ["halpern", "average"])
@pytest.mark.parametrize("n_eval", [2, 16, 128])
def test_other_evaluation_periods(B, n_eval, variant):
    P = ucgen.micro(1, B=10, L=14, G=4, T=6)
    raw, ps_o, S = oracle_pipeline(P)
    ps = B.uc_presolve(B.uc_build_lp(P))
    n, m, _, _ = B.uc_presolved_dims(ps)
    K = 3 * n_eval + 1
    ref = oracle_trace(S, [K], n_eval=n_eval, variant=variant)
    x, y, st = _device_iterates(B, ps, n, m, K, n_eval=n_eval, algorithm=variant)
    assert rel_inf(x, ref[K][0]) <= ITERATE_RTOL and rel_inf(y, ref[K][1]) <= ITERATE_RTOL


def test_warm_start_with_primal_weight_per_iterate(B):
    """A warm start (point and primal weight) follows the oracle iterate by iterate."""
    P = ucgen.tiny(2)
    raw, ps_o, S = oracle_pipeline(P)
    ref_sol = pdhg.solve_halpern(S, tol=1e-3)                  # a nearby point and its weight
    rng = np.random.default_rng(0)
    x0 = ref_sol.x * (1 + 0.01 * rng.standard_normal(ref_sol.x.size))
    y0 = ref_sol.y * (1 + 0.01 * rng.standard_normal(ref_sol.y.size))
    ks = [1, 64, 65, 130, 200]
    out = {}
    pdhg.solve_halpern(S, tol=0.0, max_iter=200, x0=x0, y0=y0, omega0=ref_sol.omega,
                       trace=lambda k, st: out.setdefault(k, (st.x.copy(), st.y.copy())), trace_iters=ks)
    ps = B.uc_presolve(B.uc_build_lp(P))
    n, m, _, _ = B.uc_presolved_dims(ps)
    for K in ks:
        res, rc = B.uc_solve(ps, tol=0.0, max_iter=K, warm_x=x0, warm_y=y0, warm_omega=ref_sol.omega)
        x, y = B.uc_get_iterate(res, 0, n, m)
        assert rel_inf(x, out[K][0]) <= ITERATE_RTOL and rel_inf(y, out[K][1]) <= ITERATE_RTOL, K


@pytest.mark.parametrize("seed", [0, 1])
def test_aggressive_presolve_parity_and_gates(B, seed):
    # the device solve of the aggressively presolved LP (doubleton equations
    # substituted) follows the oracle's PDHG on its own aggressive presolve
    # and meets the gates on the raw LP after the doubleton postsolve
    from oracle import presolve as ops
    g = golden_tiny()
    P = ucgen.tiny(seed)
    raw = olp.build_lp(P)
    ps_o = ops.presolve(raw, aggressive=True)
    S = ops.scale(ps_o.lp)
    ref = oracle_trace(S, [1, 64, 65, 200])
    ps = B.uc_presolve(B.uc_build_lp(P), aggressive=1)
    n, m, _, _ = B.uc_presolved_dims(ps)
    assert (n, m) == (ps_o.lp.n, ps_o.lp.m)
    for K in (1, 64, 65, 200):
        x, y, st = _device_iterates(B, ps, n, m, K)
        xo, yo, restarts, omega, _, _ = ref[K]
        assert st["restarts"] == restarts
        assert rel_inf(x, xo) <= ITERATE_RTOL and rel_inf(y, yo) <= ITERATE_RTOL, K
    res, rc = B.uc_solve(ps, tol=KKT_TOL)
    assert rc == B.UC_OK
    xr, yr = B.uc_get_raw_solution(res, raw.n, raw.m)
    assert max(oracle_kkt_of_raw(ps_o, xr, yr)) <= KKT_TOL * (1 + 1e-6)
    opt = g["objective_by_seed"][str(seed)]
    assert abs(raw_objective(raw, xr) - opt) / max(1.0, abs(opt)) <= OBJ_GAP_TOL


@pytest.mark.parametrize("seed", [0, 1])
def test_angle_elimination_parity_and_gates(B, seed):
    # the device solve of the angle-free LP (bus angles substituted out along a
    # spanning tree) follows the oracle's PDHG on its own angle-free presolve,
    # and after the postsolve puts the angles and the tree rows' duals back the
    # point meets the gates on the LP as built
    from oracle import presolve as ops
    g = golden_tiny()
    P = ucgen.tiny(seed)
    raw = olp.build_lp(P)
    ps_o = ops.presolve(raw, angles=True)
    S = ops.scale(ps_o.lp)
    ref = oracle_trace(S, [1, 64, 65, 200])
    ps = B.uc_presolve(B.uc_build_lp(P), eliminate_angles=1)
    n, m, _, _ = B.uc_presolved_dims(ps)
    assert (n, m) == (ps_o.lp.n, ps_o.lp.m)
    for K in (1, 64, 65, 200):
        x, y, st = _device_iterates(B, ps, n, m, K)
        xo, yo, restarts, omega, _, _ = ref[K]
        assert st["restarts"] == restarts
        assert rel_inf(x, xo) <= ITERATE_RTOL and rel_inf(y, yo) <= ITERATE_RTOL, K
    res, rc = B.uc_solve(ps, tol=KKT_TOL)
    assert rc == B.UC_OK
    r = oracle_solve(S, KKT_TOL)
    assert B.uc_get_stats(res)["iters"] == r.iters
    xr, yr = B.uc_get_raw_solution(res, raw.n, raw.m)
    # the raw LP's own KKT (the angle-free LP's rows are raw rows or implied by them)
    assert max(kkt.relative_kkt(raw, xr, yr)) <= KKT_TOL * (1 + 1e-6)
    assert max(oracle_kkt_of_raw(ps_o, xr, yr)) <= KKT_TOL * (1 + 1e-6)
    opt = g["objective_by_seed"][str(seed)]
    assert abs(raw_objective(raw, xr) - opt) / max(1.0, abs(opt)) <= OBJ_GAP_TOL
    sol = B.uc_get_solution(res, P.T, P.B, P.L, P.G)
    assert np.all(sol["theta"][:, P.ref_bus] == 0.0)


def test_long_columns_parity_batch_and_kernels(B):
    # an angle-free LP whose substituted rows put up to 55 entries in a column:
    # columns with more than 32 go last in the device layout and a warp sums
    # each (the evaluation kernel likewise).  Per-iterate parity with the
    # oracle; the period-strided and the CSR-only kernels agree bit for bit, and
    # a block-diagonal batch (the long columns in segment tables) reproduces
    # the single solve bit for bit
    from oracle import presolve as ops
    P = ucgen.batch_member(24)
    raw = olp.build_lp(P)
    ps_o = ops.presolve(raw, angles=True)
    A = ps_o.lp.A.tocsc()
    assert np.diff(A.indptr).max() > 32
    S = ops.scale(ps_o.lp)
    Ks = [1, 64, 65, 200]
    ref = oracle_trace(S, Ks)
    ps = B.uc_presolve(B.uc_build_lp(P), eliminate_angles=1)
    n, m, _, _ = B.uc_presolved_dims(ps)
    for K in Ks:
        x, y, st = _device_iterates(B, ps, n, m, K)
        xo, yo, restarts, omega, _, _ = ref[K]
        assert st["restarts"] == restarts
        assert rel_inf(x, xo) <= ITERATE_RTOL and rel_inf(y, yo) <= ITERATE_RTOL, K
        xc, yc, _ = _device_iterates(B, ps, n, m, K, spmv_kernel=1)
        np.testing.assert_array_equal(xc, x)
        np.testing.assert_array_equal(yc, y)
    small = B.uc_presolve(B.uc_build_lp(ucgen.tiny(1)), eliminate_angles=1)
    single, rc = B.uc_solve(ps, tol=KKT_TOL)
    assert rc == B.UC_OK
    batch, rc = B.uc_solve_batch([small, ps], tol=KKT_TOL)
    assert rc == B.UC_OK
    xs, ys = B.uc_get_iterate(single, 2, n, m)
    xb, yb = B.uc_get_iterate(batch[1], 2, n, m)
    np.testing.assert_array_equal(xb, xs)
    np.testing.assert_array_equal(yb, ys)
    xr, yr = B.uc_get_raw_solution(single, raw.n, raw.m)
    assert max(kkt.relative_kkt(raw, xr, yr)) <= KKT_TOL * (1 + 1e-6)


def test_long_columns_averaging_parity(B):
    # the averaging variant through the warp-per-column paths (primal kernel
    # and both candidates of the evaluation kernel) against the oracle
    from oracle import presolve as ops
    P = ucgen.batch_member(24)
    ps_o = ops.presolve(olp.build_lp(P), angles=True)
    S = ops.scale(ps_o.lp)
    Ks = [1, 64, 65, 200]
    ref = oracle_trace(S, Ks, variant="average")
    ps = B.uc_presolve(B.uc_build_lp(P), eliminate_angles=1)
    n, m, _, _ = B.uc_presolved_dims(ps)
    for K in Ks:
        x, y, st = _device_iterates(B, ps, n, m, K, algorithm="average")
        xo, yo, restarts, omega, _, _ = ref[K]
        assert st["restarts"] == restarts
        assert rel_inf(x, xo) <= ITERATE_RTOL and rel_inf(y, yo) <= ITERATE_RTOL, K
