"""Infeasibility detection on the device against the oracle: strict-model
instances (no load shedding) whose demand exceeds the generation capacity stop
with UC_EINFEASIBLE at the same iteration as the oracle, and the direction
uc_get_iterate(which = 3) returns proves infeasibility from the primal side
(the same box argument as the oracle's pins).  Feasible instances are covered
by the parity tests, which check the oracle's iteration counts."""
import numpy as np
import pytest

import ucgen
from gpu_common import KKT_TOL, oracle_pipeline
from oracle import pdhg
from test_oracle_infeasible import INFEASIBLE_CASES, _box_max

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


@pytest.mark.parametrize("lanes", [False, True])
@pytest.mark.parametrize("case", INFEASIBLE_CASES)
def test_device_detects_infeasibility_like_the_oracle(B, case, lanes):
    c = dict(case)
    P = ucgen.make_problem(c.pop("seed"), voll=0.0, **c)
    raw, ps_o, S = oracle_pipeline(P)
    ref = pdhg.solve_halpern(S, tol=KKT_TOL)
    assert ref.status == "infeasible"
    ps = B.uc_presolve(B.uc_build_lp(P))
    n, m, _, _ = B.uc_presolved_dims(ps)
    if lanes:   # two copies of the LP in one shared-matrix session
        results, rc = B.uc_solve_batch([ps, ps], tol=KKT_TOL, lanes=True)
        res = results[1]
    else:
        res, rc = B.uc_solve(ps, tol=KKT_TOL)
    assert rc == B.UC_EINFEASIBLE
    st = B.uc_get_stats(res)
    assert st["status"] == B.UC_EINFEASIBLE and st["iters"] == ref.iters
    _, y = B.uc_get_iterate(res, 3, n, m)
    np.testing.assert_allclose(y, ref.y, rtol=1e-6, atol=1e-9 * np.max(np.abs(ref.y)))
    d = B.uc_presolved_export(ps)
    import scipy.sparse as sp
    A = sp.csr_matrix((d["val"], d["colidx"], d["rowptr"]), shape=(m, n))
    # unscaled presolved LP: A_u = A_s / (D_r D_c), q_u = q_s / D_r, bounds * D_c
    Au = sp.diags(1.0 / d["Dr"]) @ A @ sp.diags(1.0 / d["Dc"])
    yu = d["Dr"] * y
    yu[d["m_eq"]:] = np.maximum(yu[d["m_eq"]:], 0.0)
    R = float(np.sum(P.x_pu * P.fmax))
    with np.errstate(invalid="ignore"):
        lu, uu = d["l"] * d["Dc"], d["u"] * d["Dc"]
    l_box = np.where(np.isfinite(lu), lu, -R)
    u_box = np.where(np.isfinite(uu), uu, R)
    assert _box_max(Au.T @ yu, l_box, u_box) < float((d["q"] / d["Dr"]) @ yu)


def test_no_direction_on_feasible_results(B):
    ps = B.uc_presolve(B.uc_build_lp(ucgen.tiny(0)))
    res, rc = B.uc_solve(ps, tol=KKT_TOL)
    assert rc == B.UC_OK
    n, m, _, _ = B.uc_presolved_dims(ps)
    with pytest.raises(B.UCError):
        B.uc_get_iterate(res, 3, n, m)
