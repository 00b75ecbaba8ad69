"""The primal-weight controller options on the device against the oracle:
the PID generalisation of PDLP's update (pw_kp, pw_ki, pw_kd) and the
residual-balance guard (pw_guard).  Both act only at restarts, in the
one-thread control kernel, so the device must take the oracle's restart
decisions and reach the oracle's weights (relative 1e-9) and iterates
(ITERATE_RTOL) at every checked step, and a full solve must take the oracle's
iterations and restarts.  The settings below change the weight from the first
or second restart on these LPs (checked against the plain rule)."""
import pytest

import ucgen
from gpu_common import ITERATE_RTOL, KKT_TOL, oracle_kkt_of_raw, oracle_pipeline, oracle_solve, oracle_trace, rel_inf

pytestmark = pytest.mark.gpu

KS = [64, 65, 128, 129, 192, 200]
SETTINGS = [((0.5, 0.05, 0.5), 0.0), ((0.5, 0.0, 0.0), 1.0), ((0.3, 0.02, 0.3), 3.0)]


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_03627_gb300 as pkg
    pkg.build()
    from paper_2607_03627_gb300 import binding
    return binding


def _problem(which):
    if which == "ragged":
        return ucgen.make_problem(7, B=37, L=53, G=11, T=5, lo=0.5, hi=0.9, noise=0.05, zero_pmin_frac=0.2)
    return ucgen.tiny(int(which[4:]))


@pytest.mark.parametrize("gains,guard", SETTINGS)
@pytest.mark.parametrize("which", ["tiny0", "ragged"])
def test_weight_control_per_iterate_parity(B, which, gains, guard):
    P = _problem(which)
    raw, ps_o, S = oracle_pipeline(P)
    ref = oracle_trace(S, KS, pw_gains=gains, pw_guard=guard)
    ps = B.uc_presolve(B.uc_build_lp(P))
    n, m, _, _ = B.uc_presolved_dims(ps)
    for K in KS:
        res, rc = B.uc_solve(ps, tol=0.0, max_iter=K, pw_gains=gains, pw_guard=guard)
        assert rc == B.UC_EITERLIMIT
        x, y = B.uc_get_iterate(res, 0, n, m)
        st = B.uc_get_stats(res)
        xo, yo, restarts, omega, _, _ = ref[K]
        assert st["restarts"] == restarts, f"restart decision differs at K={K}"
        assert st["omega"] == pytest.approx(omega, rel=1e-9)
        assert rel_inf(x, xo) <= ITERATE_RTOL and rel_inf(y, yo) <= ITERATE_RTOL


@pytest.mark.parametrize("gains,guard", SETTINGS)
@pytest.mark.parametrize("seed", range(4))
def test_weight_control_solve_takes_the_oracle_path(B, seed, gains, guard):
    P = ucgen.tiny(seed)
    raw, ps_o, S = oracle_pipeline(P)
    r = oracle_solve(S, KKT_TOL, pw_gains=gains, pw_guard=guard)
    ps = B.uc_presolve(B.uc_build_lp(P))
    res, rc = B.uc_solve(ps, tol=KKT_TOL, pw_gains=gains, pw_guard=guard)
    assert rc == B.UC_OK
    st = B.uc_get_stats(res)
    assert (st["iters"], st["restarts"]) == (r.iters, r.restarts)
    assert st["omega"] == pytest.approx(r.omega, rel=1e-9)
    xr, yr = B.uc_get_raw_solution(res, raw.n, raw.m)
    assert max(oracle_kkt_of_raw(ps_o, xr, yr)) <= KKT_TOL * (1 + 1e-6)


def test_weight_control_options_are_checked(B):
    ps = B.uc_presolve(B.uc_build_lp(ucgen.tiny(0)))
    for kw in (dict(pw_guard=0.5), dict(pw_guard=-1.0), dict(pw_guard=float("inf")),
               dict(pw_gains=(-0.1, 0.0, 0.0)), dict(pw_gains=(0.5, float("nan"), 0.0))):
        with pytest.raises(B.UCError):
            B.uc_solve(ps, tol=KKT_TOL, **kw)
