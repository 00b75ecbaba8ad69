"""The default iteration kernels, whose rows in period-strided 16-row groups
read their group's slot records instead of CSR row pointers and entries,
against the CSR-only kernels (spmv_kernel = 1).  A strided row's entry q is
its CSR entry q, so the dot products add the same terms in the same order:
every iterate, restart decision and iteration count must be identical bit for
bit -- for both algorithms, FP64 and FP32 values, any CTA size and row split,
one LP or a block-diagonal batch (whose 16-row groups may straddle two LPs),
and at the paper-scale size in the benchmarked launch shape.  Per-iterate
agreement with the oracle is in test_gpu_pdhg.py and test_gpu_fullsize.py,
which run the default kernels."""
import numpy as np
import pytest

import ucgen
from gpu_common import KKT_TOL

pytestmark = pytest.mark.gpu

STRIDED, CSR = 0, 1


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
        "small_ragged": ucgen.make_problem(7, B=37, L=53, G=11, T=5, lo=0.5, hi=0.9, noise=0.05,
                                           zero_pmin_frac=0.2),
        "mid": ucgen.make_problem(3, B=300, L=396, G=36, T=24, lo=0.5, hi=0.85, noise=0.05,
                                  zero_pmin_frac=0.1),
    }


def _same(B, ra, rb, n, m):
    sa, sb = B.uc_get_stats(ra), B.uc_get_stats(rb)
    for key in ("status", "iters", "restarts", "evals", "objective", "omega"):
        assert sa[key] == sb[key], key
    for which in (0, 1, 2):
        xa, ya = B.uc_get_iterate(ra, which, n, m)
        xb, yb = B.uc_get_iterate(rb, which, n, m)
        np.testing.assert_array_equal(xa, xb)
        np.testing.assert_array_equal(ya, yb)


def test_the_layouts_have_strided_groups(B):
    # the test LPs do exercise the strided path (and the CSR path beside it)
    for name, P in _problems().items():
        ps = B.uc_presolve(B.uc_build_lp(P))
        for tr in (False, True):
            g = B.uc_presolved_strided_groups(ps, transpose=tr)
            if name != "small_ragged":
                assert 0 < g["strided_groups"] < g["groups"], (name, tr)


@pytest.mark.parametrize("algorithm", ["halpern", "average"])
@pytest.mark.parametrize("vbits", [64, 32])
@pytest.mark.parametrize("name", ["tiny", "small_ragged", "mid"])
@pytest.mark.parametrize("K", [1, 63, 64, 65, 200])
def test_strided_iterates_equal_csr(B, name, K, vbits, algorithm):
    P = _problems()[name]
    ps = B.uc_presolve(B.uc_build_lp(P), value_bits=vbits)
    n, m, _, _ = B.uc_presolved_dims(ps)
    ra, rca = B.uc_solve(ps, tol=0.0, max_iter=K, spmv_kernel=CSR, algorithm=algorithm)
    rb, rcb = B.uc_solve(ps, tol=0.0, max_iter=K, spmv_kernel=STRIDED, algorithm=algorithm)
    assert rca == rcb == B.UC_EITERLIMIT
    _same(B, ra, rb, n, m)


@pytest.mark.parametrize("cta,rpt", [(128, 1), (256, 2), (512, 4), (128, 4)])
def test_strided_solve_equals_csr_for_any_launch_shape(B, cta, rpt):
    ps = B.uc_presolve(B.uc_build_lp(_problems()["mid"]))
    n, m, _, _ = B.uc_presolved_dims(ps)
    kw = dict(cta_rows=cta, rows_per_thread=[rpt])
    ra, rca = B.uc_solve(ps, tol=KKT_TOL, spmv_kernel=CSR, **kw)
    rb, rcb = B.uc_solve(ps, tol=KKT_TOL, spmv_kernel=STRIDED, **kw)
    assert rca == rcb == B.UC_OK
    _same(B, ra, rb, n, m)


def test_strided_batch_equals_csr_single_solves(B):
    # LPs of uneven sizes packed block-diagonally: rows of one 16-row group can
    # belong to two LPs
    pss = [B.uc_presolve(B.uc_build_lp(P)) for P in _problems().values()]
    singles = [B.uc_solve(p, tol=KKT_TOL, spmv_kernel=CSR)[0] for p in pss]
    batch, rc = B.uc_solve_batch(pss, tol=KKT_TOL, spmv_kernel=STRIDED, rows_per_thread=[1, 2, 1])
    for p, a, b in zip(pss, singles, batch):
        n, m, _, _ = B.uc_presolved_dims(p)
        _same(B, a, b, n, m)


@pytest.mark.slow
@pytest.mark.parametrize("vbits", [64, 32])
def test_strided_equals_csr_at_paper_scale(B, vbits):
    from paper_2607_03627_gb300.tune import Tuner
    ps = B.uc_presolve(B.uc_build_lp(ucgen.paper_scale(0)), value_bits=vbits)
    n, m, _, _ = B.uc_presolved_dims(ps)
    cta, rpt = Tuner().choose_pair(ps, vbits)
    kw = dict(cta_rows=cta, rows_per_thread=[rpt])
    for K in (1, 64, 200, 1000):
        ra, _ = B.uc_solve(ps, tol=0.0, max_iter=K, spmv_kernel=CSR, **kw)
        rb, _ = B.uc_solve(ps, tol=0.0, max_iter=K, spmv_kernel=STRIDED, **kw)
        _same(B, ra, rb, n, m)
