"""Crossover after the device solve (PDHG -> crossover, Sec. II-C, Alg. 1
"Solver 1"): the returned point of uc_solve on the 30-bus LPs goes through
uc_crossover; the vertex test and the simplex optimum come from the oracle."""
import numpy as np
import pytest

import ucgen
from gpu_common import KKT_TOL, golden_tiny, oracle_pipeline
from oracle import kkt, vertex

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


@pytest.mark.parametrize("seed", [0, 2])
def test_device_solve_then_crossover_is_the_simplex_vertex(B, seed):
    g = golden_tiny()
    P = ucgen.tiny(seed)
    raw, ps_o, _ = oracle_pipeline(P)
    ps = B.uc_presolve(B.uc_build_lp(P))
    res, rc = B.uc_solve(ps, tol=KKT_TOL)
    assert rc == B.UC_OK
    v, rc = B.uc_crossover(res)
    assert rc == B.UC_OK
    st = B.uc_get_stats(v)
    assert st["superbasic"] == 0 and st["iters"] > 0
    xr, yr = B.uc_get_raw_solution(v, raw.n, raw.m)
    assert vertex.is_vertex(ps_o.lp, xr[ps_o.col_map])
    opt = g["objective_by_seed"][str(seed)]
    assert abs(float(raw.c @ xr) - opt) <= 1e-9 * abs(opt)
    assert max(kkt.relative_kkt(raw, xr, yr)) <= 1e-9
    # the vertex's LMPs are the balance-row multipliers
    sol = B.uc_get_solution(v, P.T, P.B, P.L, P.G)
    assert np.all(np.isfinite(sol["lmp"]))
