"""The staged iteration kernels (persistent CTAs, chunks of matrix rows and
vectors copied into shared memory ahead of use) against the one-thread-per-row
kernels: per row they do the same operations in the same order, so every
iterate, restart decision and iteration count must be identical bit for bit,
for any number of stages, one LP or a batch, FP64 or FP32 matrix values."""
import numpy as np
import pytest

import ucgen
from gpu_common import KKT_TOL

pytestmark = pytest.mark.gpu

THREAD_PER_ROW, STAGED = 1, 2


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
        # sizes far from the 128-row chunks, zero-Pmin units
        "small_ragged": ucgen.make_problem(7, B=37, L=53, G=11, T=5, lo=0.5, hi=0.9, noise=0.05,
                                           zero_pmin_frac=0.2),
        # several hundred chunks per kernel, chunks cut by the entry cap
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


@pytest.mark.parametrize("vbits", [64, 32])
@pytest.mark.parametrize("name", ["tiny", "small_ragged", "mid"])
@pytest.mark.parametrize("K", [1, 63, 64, 65, 200])
def test_staged_iterates_equal_thread_per_row(B, name, K, vbits):
    P = _problems()[name]
    ps = B.uc_presolve(B.uc_build_lp(P), value_bits=vbits)
    n, m, _, _ = B.uc_presolved_dims(ps)
    ra, rca = B.uc_solve(ps, tol=0.0, max_iter=K, spmv_kernel=THREAD_PER_ROW)
    rb, rcb = B.uc_solve(ps, tol=0.0, max_iter=K, spmv_kernel=STAGED)
    assert rca == rcb == B.UC_EITERLIMIT
    _same(B, ra, rb, n, m)


@pytest.mark.parametrize("stages", [2, 3, 4, 8])
def test_staged_solve_independent_of_stages(B, stages):
    P = _problems()["mid"]
    ps = B.uc_presolve(B.uc_build_lp(P))
    n, m, _, _ = B.uc_presolved_dims(ps)
    ra, rca = B.uc_solve(ps, tol=KKT_TOL, spmv_kernel=THREAD_PER_ROW)
    rb, rcb = B.uc_solve(ps, tol=KKT_TOL, spmv_kernel=STAGED, stages=stages)
    assert rca == rcb == B.UC_OK
    _same(B, ra, rb, n, m)


def test_staged_without_graphs_pdl_or_reordering(B):
    P = _problems()["small_ragged"]
    ps = B.uc_presolve(B.uc_build_lp(P))
    n, m, _, _ = B.uc_presolved_dims(ps)
    for kw in (dict(use_graph=False), dict(pdl=False), dict(reorder=False)):
        ra, rca = B.uc_solve(ps, tol=KKT_TOL, spmv_kernel=THREAD_PER_ROW, **kw)
        rb, rcb = B.uc_solve(ps, tol=KKT_TOL, spmv_kernel=STAGED, **kw)
        assert rca == rcb == B.UC_OK
        _same(B, ra, rb, n, m)


def test_staged_batch_with_compaction_equals_singles(B):
    # LPs that finish at different times: the chunk lists are rebuilt for the
    # LPs still running and the results must not change
    Ps = [ucgen.tiny(0), ucgen.micro(5, B=9, L=12, G=3, T=4), ucgen.tiny(2),
          ucgen.make_problem(9, B=60, L=80, G=8, T=12, lo=0.5, hi=0.85, noise=0.05, zero_pmin_frac=0.1)]
    pss = [B.uc_presolve(B.uc_build_lp(P)) for P in Ps]
    singles = [B.uc_solve(p, tol=KKT_TOL, spmv_kernel=THREAD_PER_ROW)[0] for p in pss]
    batch, rc = B.uc_solve_batch(pss, tol=KKT_TOL, spmv_kernel=STAGED)
    assert rc == B.UC_OK
    for p, s, b in zip(pss, singles, batch):
        n, m, _, _ = B.uc_presolved_dims(p)
        _same(B, s, b, n, m)


def test_staged_option_errors(B):
    ps = B.uc_presolve(B.uc_build_lp(ucgen.tiny(0)))
    for kw in (dict(spmv_kernel=STAGED, algorithm="average"), dict(stages=1), dict(stages=9),
               dict(spmv_kernel=3)):
        with pytest.raises(B.UCError) as e:
            B.uc_solve(ps, **kw)
        assert e.value.code == B.UC_EINVAL
    res, rc = B.uc_solve(ps, tol=KKT_TOL, algorithm="average")
    assert rc == B.UC_OK
