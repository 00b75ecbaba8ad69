"""The power iteration for ||A_s||_2 run on the device (presolve option
power_device = 1) against the host power iteration and the oracle's."""
import numpy as np
import pytest

import ucgen
from gpu_common import ITERATE_RTOL, oracle_pipeline, oracle_trace, rel_inf
from oracle import lp as olp, presolve as ops

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
    yield "tiny", ucgen.tiny(0)
    yield "ragged", ucgen.make_problem(7, B=37, L=53, G=11, T=5, lo=0.5, hi=0.9, noise=0.05, zero_pmin_frac=0.2)
    yield "medium", ucgen.make_problem(2, B=400, L=530, G=48, T=24, lo=0.5, hi=0.85, noise=0.05,
                                       zero_pmin_frac=0.1)


@pytest.mark.parametrize("name,P", list(_problems()), ids=lambda v: v if isinstance(v, str) else "")
def test_device_power_iteration_matches_host_and_oracle(B, name, P):
    lp = B.uc_build_lp(P)
    h = B.uc_presolved_export(B.uc_presolve(lp))
    d = B.uc_presolved_export(B.uc_presolve(lp, power_device=1))
    # everything but the norm estimate comes from the same host code
    for k in ("rowptr", "colidx", "val", "q", "c", "l", "u", "Dr", "Dc", "omega0"):
        np.testing.assert_array_equal(d[k], h[k], err_msg=k)
    # same steps, other summation order: rounding-level differences only
    assert d["norm_A"] == pytest.approx(h["norm_A"], rel=1e-12)
    assert d["eta"] == pytest.approx(h["eta"], rel=1e-12)
    S = ops.scale(ops.presolve(olp.build_lp(P)).lp)
    assert d["eta"] == pytest.approx(S.eta, rel=1e-11)


@pytest.mark.parametrize("max_iter,tol", [(1, 1e-10), (2, 1e-10), (37, 1e-10), (500, 1e-2), (500, 1e-4)])
def test_device_power_iteration_step_count_and_stop(B, max_iter, tol):
    # the estimate rises with every product (0.985 after 50, 0.995 after 500 on the
    # 6,049-bus LP), so equal values mean the same number of products was taken
    P = ucgen.make_problem(2, B=400, L=530, G=48, T=24, lo=0.5, hi=0.85, noise=0.05, zero_pmin_frac=0.1)
    lp = B.uc_build_lp(P)
    h = B.uc_presolved_export(B.uc_presolve(lp, power_max_iter=max_iter, power_tol=tol))
    d = B.uc_presolved_export(B.uc_presolve(lp, power_max_iter=max_iter, power_tol=tol, power_device=1))
    assert d["norm_A"] == pytest.approx(h["norm_A"], rel=1e-13)


def test_device_power_iteration_per_iterate_parity(B):
    P = ucgen.tiny(0)
    _, _, S = oracle_pipeline(P)
    ks = [1, 64, 65, 200]
    ref = oracle_trace(S, ks)
    ps = B.uc_presolve(B.uc_build_lp(P), power_device=1)
    n, m, _, _ = B.uc_presolved_dims(ps)
    for K in ks:
        res, rc = B.uc_solve(ps, tol=0.0, max_iter=K)
        assert rc == B.UC_EITERLIMIT
        x, y = B.uc_get_iterate(res, 0, n, m)
        xo, yo = ref[K][0], ref[K][1]
        assert rel_inf(x, xo) <= ITERATE_RTOL and rel_inf(y, yo) <= ITERATE_RTOL, K


def test_device_power_iteration_full_size(B):
    lp = B.uc_build_lp(ucgen.paper_scale(0))
    h = B.uc_presolved_export(B.uc_presolve(lp))
    d = B.uc_presolved_export(B.uc_presolve(lp, power_device=1))
    assert d["norm_A"] == pytest.approx(h["norm_A"], rel=1e-12)
    assert 0.99 < d["norm_A"] <= 1.0   # below the Schur bound of the scaled matrix
