"""Failure statuses, each caused on the host (no GPU fault, trap or hang):
a NaN in the warm start -> UC_ENUMERIC from the device evaluation; a tiny
timeout -> UC_ETIMEOUT at the next replay boundary; a set cancel flag ->
UC_ECANCELLED; invalid options are rejected before any device work."""
import ctypes

import numpy as np
import pytest

import ucgen

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


@pytest.fixture(scope="module")
def ps(B):
    return B.uc_presolve(B.uc_build_lp(ucgen.tiny(2)))


def test_nan_warm_start_reports_numeric(B, ps):
    n, m, _, _ = B.uc_presolved_dims(ps)
    y = np.zeros(m)
    y[3] = np.nan
    res, rc = B.uc_solve(ps, tol=1e-4, warm_y=y)
    assert rc == -7                                  # UC_ENUMERIC
    assert B.uc_get_stats(res)["iters"] == 0


def test_timeout_stops_at_a_replay_boundary(B, ps):
    res, rc = B.uc_solve(ps, tol=1e-12, timeout_ms=1e-3)
    assert rc == B.UC_ETIMEOUT
    it = B.uc_get_stats(res)["iters"]
    assert it % 64 == 0 and 0 < it <= 3 * 64


def test_cancel_flag(B, ps):
    flag = ctypes.c_int(1)
    res, rc = B.uc_solve(ps, tol=1e-12, cancel=flag)
    assert rc == B.UC_ECANCELLED


def test_invalid_options_rejected(B, ps):
    with pytest.raises(B.UCError, match="n_eval"):
        B.uc_solve(ps, n_eval=3)
    with pytest.raises(B.UCError, match="rows_per_thread"):
        B.uc_solve(ps, rows_per_thread=[3])
    with pytest.raises(B.UCError, match="cta_rows"):
        B.uc_solve(ps, cta_rows=100)
