"""The concurrent solve of Alg. 1 (Sec. II-C): device PDHG and host simplex
at once on one LP, the first optimal arm stops the other.

* 30-bus LP: the device arm ends first (tens of milliseconds against the dense
  simplex's seconds); its result is the plain uc_solve result bit for bit and
  the host arm is stopped early.
* A micro LP with a device tolerance it cannot reach: the host simplex wins
  with the simplex optimum at a vertex, and the device arm stops at its next
  replay boundary instead of running to its iteration limit.
"""
import time

import numpy as np
import pytest

import ucgen
from gpu_common import KKT_TOL
from oracle import lp as olp, presolve as ops, simplex, vertex

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


def test_device_arm_wins_on_the_30_bus_lp(B):
    ps = B.uc_presolve(B.uc_build_lp(ucgen.tiny(0)))
    n, m, _, _ = B.uc_presolved_dims(ps)
    t0 = time.perf_counter()
    res, rc, winner = B.uc_solve_concurrent(ps, tol=KKT_TOL)
    wall = time.perf_counter() - t0
    assert rc == B.UC_OK and winner == 0
    alone, _ = B.uc_solve(ps, tol=KKT_TOL)
    for which in (0, 2):
        xa, ya = B.uc_get_iterate(alone, which, n, m)
        xb, yb = B.uc_get_iterate(res, which, n, m)
        np.testing.assert_array_equal(xa, xb)
        np.testing.assert_array_equal(ya, yb)
    assert wall < 10.0          # the host simplex (about 25 s alone here) was stopped


def test_host_arm_wins_when_the_device_cannot_finish(B):
    P = ucgen.micro(2, B=5, L=6, G=3, T=3)
    raw = olp.build_lp(P)
    ps_o = ops.presolve(raw)
    ref = simplex.solve_lp(raw)
    ps = B.uc_presolve(B.uc_build_lp(P))
    t0 = time.perf_counter()
    res, rc, winner = B.uc_solve_concurrent(ps, tol=1e-15, max_iter=50_000_000)
    wall = time.perf_counter() - t0
    assert rc == B.UC_OK and winner == 1
    xr, yr = B.uc_get_raw_solution(res, raw.n, raw.m)
    assert abs(float(raw.c @ xr) - ref.obj) <= 1e-9 * abs(ref.obj)
    assert vertex.is_vertex(ps_o.lp, xr[ps_o.col_map])
    assert wall < 30.0          # 50 M device iterations would take minutes
