"""Primal feasibility polishing on the device (uc_solve with polish = 1)
against the oracle's polish_primal: the paper runs its PDHG with an absolute
feasibility tolerance of 1e-5 beside the 1e-4 convergence tolerance (Sec.
II-D).  After the main solve (same iterations as the oracle's), the
polishing phase must take the oracle's number of iterations, end at the
oracle's polished point (ITERATE_RTOL), and leave every row of the raw LP
violated by at most 1e-5 (checked with the oracle's absolute-violation
figure) while the objective stays within the 1e-4 gap of the simplex."""
import numpy as np
import pytest

import ucgen
from gpu_common import (ITERATE_RTOL, KKT_TOL, OBJ_GAP_TOL, golden_tiny, oracle_pipeline, raw_objective,
                        rel_inf)
from oracle import kkt, pdhg, presolve as ops

pytestmark = pytest.mark.gpu

ABS_TOL = 1e-5


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_03627_gb300 as pkg
    pkg.build()
    from paper_2607_03627_gb300 import binding
    return binding


@pytest.mark.parametrize("seed", range(4))
def test_polish_matches_oracle_and_meets_the_absolute_tolerance(B, seed):
    g = golden_tiny()
    P = ucgen.tiny(seed)
    raw, ps_o, S = oracle_pipeline(P)
    main = pdhg.solve_halpern(S, tol=KKT_TOL)
    pol = pdhg.polish_primal(S, main.x, ABS_TOL, omega0=main.omega)
    assert pol.status == "optimal"
    ps = B.uc_presolve(B.uc_build_lp(P))
    n, m, _, _ = B.uc_presolved_dims(ps)
    res, rc = B.uc_solve(ps, tol=KKT_TOL, polish=True, tol_abs_feas=ABS_TOL)
    assert rc == B.UC_OK
    st = B.uc_get_stats(res)
    assert st["iters"] == main.iters
    assert st["abs_primal_unpolished"] > ABS_TOL          # there was something to polish
    assert st["polish_iters"] == pol.iters
    x, y = B.uc_get_iterate(res, 2, n, m)
    assert rel_inf(x, pol.x) <= ITERATE_RTOL
    assert rel_inf(y, main.y) <= ITERATE_RTOL              # the dual is the main solve's
    xr, yr = B.uc_get_raw_solution(res, raw.n, raw.m)
    assert kkt.abs_primal_inf(raw, xr) <= ABS_TOL * (1 + 1e-6)
    assert st["abs_primal"] <= ABS_TOL
    opt = g["objective_by_seed"][str(seed)]
    assert abs(raw_objective(raw, xr) - opt) / max(1.0, abs(opt)) <= OBJ_GAP_TOL
    # the reported KKT figures are those of the combined point
    rel = kkt.relative_kkt(ps_o.lp, xr[ps_o.col_map], yr[ps_o.row_map])
    np.testing.assert_allclose([st["rel_primal"], st["rel_dual"], st["rel_gap"]], rel, rtol=1e-6, atol=1e-12)


def test_polish_skips_points_already_within_the_tolerance(B):
    P = ucgen.tiny(0)
    ps = B.uc_presolve(B.uc_build_lp(P))
    res, rc = B.uc_solve(ps, tol=KKT_TOL, polish=True, tol_abs_feas=1.0)
    assert rc == B.UC_OK
    st = B.uc_get_stats(res)
    assert st["polish_iters"] == 0 and st["abs_primal"] == st["abs_primal_unpolished"] <= 1.0


def test_polish_options_are_checked(B):
    ps = B.uc_presolve(B.uc_build_lp(ucgen.tiny(0)))
    for kw in (dict(algorithm="average"), dict(tol_abs_feas=0.0), dict(polish_max_iter=-1)):
        with pytest.raises(B.UCError):
            B.uc_solve(ps, tol=KKT_TOL, polish=True, **kw)


@pytest.mark.slow
def test_polish_at_paper_scale(B):
    P = ucgen.paper_scale(0)
    raw, ps_o, S = oracle_pipeline(P)
    ps = B.uc_presolve(B.uc_build_lp(P), power_device=1)
    res, rc = B.uc_solve(ps, tol=KKT_TOL, polish=True, tol_abs_feas=ABS_TOL)
    assert rc == B.UC_OK
    st = B.uc_get_stats(res)
    xr, yr = B.uc_get_raw_solution(res, raw.n, raw.m)
    assert kkt.abs_primal_inf(raw, xr) <= ABS_TOL * (1 + 1e-6)
    rel = kkt.relative_kkt(ps_o.lp, xr[ps_o.col_map], yr[ps_o.row_map])
    print(f"paper scale: {st['iters']} + {st['polish_iters']} polish iterations, abs violation "
          f"{st['abs_primal_unpolished']:.2e} -> {st['abs_primal']:.2e}, rel KKT {max(rel):.2e}")
