"""GPU tests of batching (row split independence, tuner) and of the server
(each request's result is the same alone and in the mix)."""
import numpy as np
import pytest

import ucgen
from gpu_common import KKT_TOL, oracle_kkt_of_raw, oracle_pipeline

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


def test_batch_row_split_and_compaction_do_not_change_results(B):
    Ps = [ucgen.tiny(0), ucgen.micro(5, B=9, L=12, G=3, T=4), ucgen.tiny(2),
          ucgen.make_problem(9, B=60, L=80, G=8, T=12, lo=0.5, hi=0.85, noise=0.05, zero_pmin_frac=0.1)]
    pss = [B.uc_presolve(B.uc_build_lp(P)) for P in Ps]
    singles = [B.uc_solve(p, tol=KKT_TOL)[0] for p in pss]
    batch, rc = B.uc_solve_batch(pss, tol=KKT_TOL, rows_per_thread=[4, 2, 1, 2], cta_rows=128)
    assert rc == B.UC_OK
    for p, s, b in zip(pss, singles, batch):
        n, m, _, _ = B.uc_presolved_dims(p)
        for which in (0, 2):
            xs, ys = B.uc_get_iterate(s, which, n, m)
            xb, yb = B.uc_get_iterate(b, which, n, m)
            np.testing.assert_array_equal(xb, xs)
            np.testing.assert_array_equal(yb, ys)


def test_solve_batch_with_tuner(B, tmp_path):
    from paper_2607_03627_gb300.batch import presolve_all, solve_batch
    from paper_2607_03627_gb300.tune import Tuner
    Ps = [ucgen.make_problem(s, B=40 + 20 * s, L=55 + 26 * s, G=5 + s, T=12, lo=0.5, hi=0.85, noise=0.05,
                             zero_pmin_frac=0.1) for s in range(5)]
    pss = presolve_all(Ps, value_bits=32)
    tuner = Tuner(cache_path=str(tmp_path / "tune.json"), trial_replays=2)
    results, info = solve_batch(pss, tol=KKT_TOL, tuner=tuner, value_bits=32)
    assert set(info["rows_per_thread"]) <= {1, 2, 4}
    assert (tmp_path / "tune.json").exists()
    for P, (res, rc) in zip(Ps, results):
        assert rc == B.UC_OK
        raw, ps_o, _ = oracle_pipeline(P)
        xr, yr = B.uc_get_raw_solution(res, raw.n, raw.m)
        assert max(oracle_kkt_of_raw(ps_o, xr, yr)) <= 1.1 * KKT_TOL   # FP32-stored matrix


def test_presolve_reuse_matches_full_presolve(B):
    base = ucgen.tiny(3)
    ps0 = B.uc_presolve(B.uc_build_lp(base))
    Q = ucgen.served_request(base, 1, 7)
    full = B.uc_presolved_export(B.uc_presolve(B.uc_build_lp(Q)))
    re = B.uc_presolved_export(B.uc_presolve_reuse(ps0, B.uc_build_lp(Q)))
    for k in ("rowptr", "colidx", "val", "q", "c", "l", "u", "Dr", "Dc", "col_map", "row_map"):
        np.testing.assert_array_equal(re[k], full[k], err_msg=k)
    for k in ("eta", "omega0", "q_inf", "c_inf", "obj_const"):
        assert re[k] == full[k], k
    other = ucgen.tiny(4)                         # another grid: must be refused
    with pytest.raises(B.UCError, match="matrix differs"):
        B.uc_presolve_reuse(ps0, B.uc_build_lp(other))


@pytest.mark.parametrize("slots", [3, 4])   # block-diagonal slots; a shared-matrix (lanes) session
def test_server_results_same_alone_and_in_the_mix(B, slots):
    from paper_2607_03627_gb300.serve import Request, Server
    base = ucgen.tiny(0)
    reqs = [Request(rid=r, problem=ucgen.served_request(base, 0, r), arrival=0.05 * r) for r in range(8)]
    srv = Server(base, slots=slots, tol=KKT_TOL, keep_solutions=True, replays_per_step=2, presolve_workers=4)
    m = srv.serve(reqs, realtime=False)
    srv.close()
    assert m["all_optimal"] and m["slots"] == slots and m["warm_started"] >= 1
    # a warm start that fails is solved again cold (its start fields then say cold)
    assert all(r.start_y is None for r in reqs if r.retried_cold)
    assert m["lanes"] == (slots == 4)
    assert any(r.admitted > 0 and r.slot >= 0 for r in reqs)
    base_ps = B.uc_presolve(B.uc_build_lp(base))
    for r in reqs:
        ps = B.uc_presolve_reuse(base_ps, B.uc_build_lp(r.problem))
        res, rc = B.uc_solve(ps, tol=KKT_TOL, warm_x=r.start_x, warm_y=r.start_y, warm_omega=r.start_omega)
        assert rc == B.UC_OK
        n, m_, _, _ = B.uc_presolved_dims(ps)
        x, y = B.uc_get_iterate(res, 2, n, m_)
        np.testing.assert_array_equal(x, r.x)          # identical iterates: same arithmetic
        np.testing.assert_array_equal(y, r.y)
        assert B.uc_get_stats(res)["iters"] == r.iters
        raw, ps_o, _ = oracle_pipeline(r.problem)
        xr, yr = B.uc_get_raw_solution(res, raw.n, raw.m)
        assert max(oracle_kkt_of_raw(ps_o, xr, yr)) <= KKT_TOL * (1 + 1e-6)


def test_server_respects_hbm_budget(B):
    from paper_2607_03627_gb300.serve import Server
    base = ucgen.tiny(1)
    probe = Server(base, slots=1)
    per = probe.bytes_per_slot
    probe.close()
    srv = Server(base, slots=8, hbm_budget_gb=2.5 * per / 1e9)
    assert srv.slots == 2
    srv.close()


@pytest.mark.parametrize("vbits", [64, 32])
@pytest.mark.parametrize("K", [1, 64, 65, 200])
def test_two_rows_per_thread_equal_one_row(B, K, vbits):
    # the row split changes which thread does a row, never its arithmetic
    for P in (ucgen.tiny(0), ucgen.make_problem(3, B=300, L=396, G=36, T=24, lo=0.5, hi=0.85, noise=0.05,
                                                zero_pmin_frac=0.1)):
        ps = B.uc_presolve(B.uc_build_lp(P), value_bits=vbits)
        n, m, _, _ = B.uc_presolved_dims(ps)
        for cta in (128, 256):
            r1, rc1 = B.uc_solve(ps, tol=0.0, max_iter=K, rows_per_thread=[1], cta_rows=cta)
            r2, rc2 = B.uc_solve(ps, tol=0.0, max_iter=K, rows_per_thread=[2], cta_rows=cta)
            assert rc1 == rc2 == B.UC_EITERLIMIT
            for which in (0, 1, 2):
                x1, y1 = B.uc_get_iterate(r1, which, n, m)
                x2, y2 = B.uc_get_iterate(r2, which, n, m)
                np.testing.assert_array_equal(x1, x2)
                np.testing.assert_array_equal(y1, y2)
            s1, s2 = B.uc_get_stats(r1), B.uc_get_stats(r2)
            assert (s1["restarts"], s1["omega"]) == (s2["restarts"], s2["omega"])


def _mixed_requests():
    from paper_2607_03627_gb300.serve import Request
    a, b = ucgen.tiny(0), ucgen.tiny(4)           # two grids of the same size class
    c = ucgen.make_problem(7, B=37, L=53, G=11, T=5, lo=0.5, hi=0.9, noise=0.05, zero_pmin_frac=0.2)
    probs = [ucgen.served_request(a, 0, 0), b, c, ucgen.served_request(a, 0, 1), ucgen.served_request(b, 0, 2), c]
    return [Request(rid=i, problem=P, arrival=0.02 * i) for i, P in enumerate(probs)]


def test_mixed_server_results_same_alone_and_in_the_mix(B):
    from paper_2607_03627_gb300.serve import MixedServer
    reqs = _mixed_requests()
    srv = MixedServer(max_active=3, tol=KKT_TOL, keep_solutions=True)
    m = srv.serve(reqs)
    srv.close()
    assert m["all_optimal"] and m["peak_active"] >= 2          # grids of different sizes overlapped
    for r in reqs:
        ps = B.uc_presolve(B.uc_build_lp(r.problem))
        res, rc = B.uc_solve(ps, tol=KKT_TOL)
        assert rc == B.UC_OK
        n, m_, _, _ = B.uc_presolved_dims(ps)
        x, y = B.uc_get_iterate(res, 2, n, m_)
        np.testing.assert_array_equal(x, r.x)
        np.testing.assert_array_equal(y, r.y)
        assert B.uc_get_stats(res)["iters"] == r.iters
        raw, ps_o, _ = oracle_pipeline(r.problem)
        xr, yr = B.uc_get_raw_solution(res, raw.n, raw.m)
        assert max(oracle_kkt_of_raw(ps_o, xr, yr)) <= KKT_TOL * (1 + 1e-6)


def test_mixed_server_admits_by_hbm_budget(B):
    from paper_2607_03627_gb300.serve import MixedServer, session_bytes_estimate
    reqs = _mixed_requests()
    big = max(session_bytes_estimate(B.uc_presolve(B.uc_build_lp(r.problem))) for r in reqs)
    srv = MixedServer(max_active=4, hbm_budget_gb=big / 1e9, tol=KKT_TOL)
    m = srv.serve(reqs)
    srv.close()
    assert m["all_optimal"] and m["peak_active"] == 1        # the budget holds one session at a time
    # and the estimate is an upper bound on what a session takes
    ps = B.uc_presolve(B.uc_build_lp(reqs[0].problem))
    sess = B.Session([ps], tol=KKT_TOL)
    assert sess.device_bytes() <= session_bytes_estimate(ps)
    sess.close()


MID_SEEDS = [5, 6, 11, 18, 27, 40, 52, 57]   # batch recipe, 456 to 1,438 buses, T 24 and 48


@pytest.mark.slow
def test_batch_of_uneven_mid_size_lps_meets_the_kkt_gate(B):
    # eight LPs of the batch recipe (300-1,500 buses) in one block-diagonal
    # session with uneven row splits: every result's KKT is re-evaluated by the
    # oracle on its own presolve, and one of them equals its single solve bit for bit
    probs = [ucgen.batch_member(s) for s in MID_SEEDS]
    pss = [B.uc_presolve(B.uc_build_lp(P)) for P in probs]
    results, rc = B.uc_solve_batch(pss, tol=KKT_TOL, rows_per_thread=[1, 2, 1, 4, 2, 1, 2, 1])
    assert rc == B.UC_OK
    for P, r in zip(probs, results):
        raw, ps_o, _ = oracle_pipeline(P)
        xr, yr = B.uc_get_raw_solution(r, raw.n, raw.m)
        assert max(oracle_kkt_of_raw(ps_o, xr, yr)) <= KKT_TOL * (1 + 1e-6), P.name
        sol = B.uc_get_solution(r, P.T, P.B, P.L, P.G)
        bal = sol["p"].sum(axis=1) + sol["shed"].sum(axis=1) - P.load.sum(axis=1)
        assert np.max(np.abs(bal)) <= P.B * KKT_TOL * (1 + np.max(np.abs(ps_o.lp.q))), P.name
    n, m, _, _ = B.uc_presolved_dims(pss[3])
    single, _ = B.uc_solve(pss[3], tol=KKT_TOL)
    for which in (0, 2):
        xa, ya = B.uc_get_iterate(single, which, n, m)
        xb, yb = B.uc_get_iterate(results[3], which, n, m)
        np.testing.assert_array_equal(xa, xb)
        np.testing.assert_array_equal(ya, yb)
