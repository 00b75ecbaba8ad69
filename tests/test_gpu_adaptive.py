"""PDLP's adaptive step size (averaging variant) on the device against the
oracle: per-attempt iterates, the accept / reject sequence, and solves to the
paper's tolerance."""
import numpy as np
import pytest

import ucgen
from gpu_common import (ITERATE_RTOL, KKT_TOL, OBJ_GAP_TOL, golden_tiny, oracle_kkt_of_raw,
                        oracle_pipeline, raw_objective, rel_inf)
from oracle import pdhg

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


def _problems():
    return {
        "tiny": ucgen.tiny(0),
        "ragged": ucgen.make_problem(7, B=37, L=53, G=11, T=5, lo=0.5, hi=0.9, noise=0.05, zero_pmin_frac=0.2),
        # rejects its 3rd attempt
        "reject3": ucgen.make_problem(6, B=20, L=26, G=5, T=8, lo=0.4, hi=0.8, noise=0.05, zero_pmin_frac=0.25),
        # rejects its 66th attempt, right after an evaluation
        "reject66": ucgen.micro(5, B=5, L=6, G=2, T=3),
    }


KS = [1, 2, 3, 4, 5, 17, 63, 64, 65, 66, 67, 100, 128]


def _oracle_traces(S, ks):
    """{exact_sums: {k: (x, y, rejected, restarts, omega)}} for the oracle with
    numpy's sums and with correctly rounded sums in the step bound."""
    out = {}
    for exact in (False, True):
        d = {}
        def rec(k, st, d=d):
            d[k] = (st.x.copy(), st.y.copy(), st.k - st.accepted, st.restarts, st.omega)
        pdhg.solve(S, tol=0.0, max_iter=max(ks), adaptive=True, exact_sums=exact, trace=rec, trace_iters=ks)
        out[exact] = d
    return out


# Tolerance.  The step bound eta_bar divides by |dy^T A dx|, a sum that cancels,
# and each attempt's step follows from the last one's bound, so rounding alone
# moves the trajectory, and more with every attempt: the oracle with numpy's
# sums and with correctly rounded sums differ by ~1e-14 after 64 attempts and
# ~1e-5 after 200 on the 30-bus LP.  Per attempt, the device must stay within
# max(1e-9, 10 x that spread), at checkpoints where the spread is still small.
@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("which", ["tiny", "ragged", "reject3", "reject66"])
def test_adaptive_per_attempt_parity(B, which, use_graph):
    P = _problems()[which]
    _, _, S = oracle_pipeline(P)
    tr = _oracle_traces(S, KS)
    ps = B.uc_presolve(B.uc_build_lp(P))
    n, m, _, _ = B.uc_presolved_dims(ps)
    for K in KS:
        xo, yo, rejected, restarts, omega = tr[False][K]
        xe, ye, rej_e, _, _ = tr[True][K]
        spread = max(rel_inf(xe, xo), rel_inf(ye, yo))
        assert spread <= 1e-8 and rej_e == rejected, f"checkpoint K={K} is past the well-conditioned range"
        tol = max(ITERATE_RTOL, 10.0 * spread)
        res, rc = B.uc_solve(ps, tol=0.0, max_iter=K, algorithm="average", adaptive_step=True,
                             use_graph=use_graph)
        assert rc == B.UC_EITERLIMIT
        st = B.uc_get_stats(res)
        x, y = B.uc_get_iterate(res, 0, n, m)
        assert st["iters"] == K
        assert st["rejected_steps"] == rejected, f"accept / reject sequence differs by K={K}"
        assert st["restarts"] == restarts, f"restart decision differs at K={K}"
        assert rel_inf(x, xo) <= tol, (K, rel_inf(x, xo), tol)
        assert rel_inf(y, yo) <= tol, (K, rel_inf(y, yo), tol)
        assert st["omega"] == pytest.approx(omega, rel=max(1e-9, 10.0 * spread))
    if which.startswith("reject"):
        assert tr[False][max(KS)][2] > 0


@pytest.mark.parametrize("seed", range(3))
def test_adaptive_solve_meets_gates(B, seed):
    g = golden_tiny()
    P = ucgen.tiny(seed)
    raw, ps_o, S = oracle_pipeline(P)
    ps = B.uc_presolve(B.uc_build_lp(P))
    res, rc = B.uc_solve(ps, tol=KKT_TOL, algorithm="average", adaptive_step=True)
    assert rc == B.UC_OK
    st = B.uc_get_stats(res)
    xr, yr = B.uc_get_raw_solution(res, raw.n, raw.m)
    assert max(oracle_kkt_of_raw(ps_o, xr, yr)) <= KKT_TOL * (1 + 1e-6)
    opt = g["objective_by_seed"][str(seed)]
    assert abs(raw_objective(raw, xr) - opt) / max(1.0, abs(opt)) <= OBJ_GAP_TOL
    # the trajectory depends on rounding (see above), so the iteration count is
    # not compared with the oracle's; the gates above are the parity here


def test_adaptive_average_and_fp32_values(B):
    # the returned average is the step-weighted one; FP32 values run the same rule
    P = _problems()["reject3"]
    _, _, S = oracle_pipeline(P)
    K = 100   # past the evaluation (and restart) after attempt 64
    st_o = pdhg.solve(S, tol=0.0, max_iter=K, adaptive=True).state
    assert st_o.accepted < K and st_o.restarts > 0
    lp = B.uc_build_lp(P)
    ps = B.uc_presolve(lp)
    n, m, _, _ = B.uc_presolved_dims(ps)
    res, rc = B.uc_solve(ps, tol=0.0, max_iter=K, algorithm="average", adaptive_step=True)
    assert rc == B.UC_EITERLIMIT
    xa, ya = B.uc_get_iterate(res, 1, n, m)
    assert rel_inf(xa, st_o.x_sum / st_o.w_sum) <= 1e-8
    assert rel_inf(ya, st_o.y_sum / st_o.w_sum) <= 1e-8
    r32, rc32 = B.uc_solve(B.uc_presolve(lp, value_bits=32), tol=KKT_TOL, algorithm="average",
                           adaptive_step=True)
    assert rc32 == B.UC_OK


def test_adaptive_option_is_checked(B):
    ps = B.uc_presolve(B.uc_build_lp(ucgen.tiny(0)))
    with pytest.raises(B.UCError, match="adaptive_step"):
        B.uc_solve(ps, tol=KKT_TOL, adaptive_step=True)              # Halpern
    with pytest.raises(B.UCError, match="adaptive_step"):
        B.uc_solve_batch([ps, ps], tol=KKT_TOL, algorithm="average", adaptive_step=True)
