"""Shared-matrix ("lanes") sessions: 2 or 4 LPs with one scaled matrix (load
variants of one grid, presolved with uc_presolve_reuse), the matrix stored
once and the vectors interleaved.  Per LP the arithmetic is that of a solve of
that LP alone, operation for operation and in the same order, so every
iterate, restart decision and iteration count must be identical bit for bit
to the separate solves, whatever the other lanes do."""
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


def _requests(B, base, count, vbits=64):
    base_ps = B.uc_presolve(B.uc_build_lp(base), value_bits=vbits)
    probs = [ucgen.served_request(base, 1, r) for r in range(count)]
    return probs, [B.uc_presolve_reuse(base_ps, B.uc_build_lp(P)) for P in probs]


def _same(B, ra, rb, n, m):
    sa, sb = B.uc_get_stats(ra), B.uc_get_stats(rb)
    for key in ("status", "iters", "restarts", "evals", "objective", "omega", "rel_primal", "rel_dual", "rel_gap"):
        assert sa[key] == sb[key], key
    for which in (0, 1, 2):
        xa, ya = B.uc_get_iterate(ra, which, n, m)
        xb, yb = B.uc_get_iterate(rb, which, n, m)
        np.testing.assert_array_equal(xa, xb)
        np.testing.assert_array_equal(ya, yb)


@pytest.mark.parametrize("vbits", [64, 32])
@pytest.mark.parametrize("lanes", [2, 4])
def test_lanes_solve_equals_separate_solves(B, lanes, vbits):
    base = ucgen.make_problem(11, B=60, L=80, G=8, T=12, lo=0.5, hi=0.85, noise=0.05, zero_pmin_frac=0.1)
    probs, pss = _requests(B, base, lanes, vbits)
    n, m, _, _ = B.uc_presolved_dims(pss[0])
    singles = [B.uc_solve(p, tol=KKT_TOL) for p in pss]
    batch, rc = B.uc_solve_batch(pss, tol=KKT_TOL, lanes=True)
    assert rc == B.UC_OK
    iters = set()
    for (s, rcs), b, P in zip(singles, batch, probs):
        assert rcs == B.UC_OK
        _same(B, s, b, n, m)
        iters.add(B.uc_get_stats(b)["iters"])
        raw, ps_o, _ = oracle_pipeline(P)
        xr, yr = B.uc_get_raw_solution(b, raw.n, raw.m)
        assert max(oracle_kkt_of_raw(ps_o, xr, yr)) <= (1 + 1e-6 if vbits == 64 else 1.1) * KKT_TOL
    assert len(iters) > 1   # the lanes finish at different times


@pytest.mark.parametrize("K", [1, 64, 65, 200])
def test_lanes_iterates_equal_separate_solves(B, K):
    base = ucgen.tiny(4)
    _, pss = _requests(B, base, 4)
    n, m, _, _ = B.uc_presolved_dims(pss[0])
    batch, rc = B.uc_solve_batch(pss, tol=0.0, max_iter=K, lanes=True)
    assert rc == B.UC_EITERLIMIT
    for p, b in zip(pss, batch):
        s, rcs = B.uc_solve(p, tol=0.0, max_iter=K)
        assert rcs == B.UC_EITERLIMIT
        _same(B, s, b, n, m)


def test_lanes_session_refill_and_warm_start(B):
    """A lane is harvested, refilled with another request (new right-hand side
    and bounds, warm-started) and reset while the other lane keeps iterating;
    both results equal separate solves."""
    base = ucgen.tiny(5)
    probs, pss = _requests(B, base, 3)
    n, m, _, _ = B.uc_presolved_dims(pss[0])
    sess = B.Session([pss[0], pss[1]], tol=KKT_TOL, lanes=True)
    sess.reset(-1)
    while sess.status(0) == 2 and sess.status(1) == 2:
        sess.run(1)
    first = 0 if sess.status(0) != 2 else 1
    res_first, rc = sess.result(first)
    assert rc == B.UC_OK
    _same(B, B.uc_solve(pss[first], tol=KKT_TOL)[0], res_first, n, m)
    # refill the finished lane with request 2, warm-started from request `first`'s duals and weight
    xw, yw = B.uc_get_iterate(res_first, 2, n, m)
    omega = B.uc_get_stats(res_first)["omega"]
    sess.update_lp(first, pss[2])
    sess.set_start(first, None, yw, omega)
    sess.reset(first)
    sess.run()
    other = 1 - first
    for lane, p, kw in ((first, pss[2], dict(warm_y=yw, warm_omega=omega)), (other, pss[other], {})):
        res, rc = sess.result(lane)
        assert rc == B.UC_OK
        _same(B, B.uc_solve(p, tol=KKT_TOL, **kw)[0], res, n, m)
    sess.close()


def test_lanes_option_errors(B):
    base = ucgen.tiny(6)
    _, pss = _requests(B, base, 3)
    other = B.uc_presolve(B.uc_build_lp(ucgen.tiny(7)))
    for lps, kw in (([pss[0], pss[1], pss[2]], {}),               # 3 LPs
                    ([pss[0], other], {}),                         # different matrices
                    ([pss[0], pss[1]], dict(algorithm="average")),
                    ([pss[0], pss[1]], dict(spmv_kernel=2))):
        with pytest.raises(B.UCError) as e:
            B.uc_solve_batch(lps, tol=KKT_TOL, lanes=True, **kw)
        assert e.value.code == B.UC_EINVAL
