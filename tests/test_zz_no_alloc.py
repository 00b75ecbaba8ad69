"""The allocation-free KKT entry point (uc_kkt_noalloc) against the oracle's
KKT definitions and against the solver's own evaluation.

uc_kkt_noalloc serves callers that must not allocate device memory: a process
whose device memory is reserved up front by its own pool allocator, or a
latency-bound loop that must not enter the allocator.  It keeps its scratch in
a fixed array of the library, shared by every call.  Here, on LPs the oracle
presolved and scaled (copied into device memory by the test):

* its eight outputs equal the oracle's relative KKT parts, weighted KKT,
  objectives and unscaled primal residual of the same point, on the 30-bus LP
  (a handful of CTAs) and on the 6,049-bus LP (about 1,860 CTAs, so the
  finishing kernel's loop over the CTA records takes several passes);
* at the solver's returned point they also equal what uc_solve reported;
* two calls in a row give the same bits (the second reuses the scratch the
  first left behind), and after the first call on the device the free device
  memory does not change;
* a NaN in the point comes out as NaN, as in the solver's evaluation;
* sizes beyond the fixed array, up to INT_MAX rows and columns, are refused.
"""
import numpy as np
import pytest

import ucgen
from gpu_common import ITERATE_RTOL, KKT_TOL, oracle_pipeline
from oracle import kkt, pdhg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_03627_gb300 as pkg
    pkg.build()
    from paper_2607_03627_gb300 import binding
    return binding


class DeviceLp:
    """The oracle's scaled LP copied into device memory (torch tensors), and
    the uc_device_lp that points at it."""

    def __init__(self, B, S):
        import torch
        dev = torch.device("cuda", 0)
        t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
        AT = S.A.T.tocsr()
        AT.sort_indices()
        self.keep = dict(A_rowptr=t(S.A.indptr, torch.int32), A_colidx=t(S.A.indices, torch.int32),
                         A_val=t(S.A.data, torch.float64), AT_rowptr=t(AT.indptr, torch.int32),
                         AT_colidx=t(AT.indices, torch.int32), AT_val=t(AT.data, torch.float64),
                         c=t(S.c, torch.float64), l=t(S.l, torch.float64), u=t(S.u, torch.float64),
                         Dc=t(S.Dc, torch.float64), q=t(S.q, torch.float64), Dr=t(S.Dr, torch.float64))
        m, n = S.A.shape
        self.lp = B.uc_device_lp(n=n, m=m, m_eq=S.m_eq, q_inf=S.q_inf_unscaled, c_inf=S.c_inf_unscaled,
                                 **{k: v.data_ptr() for k, v in self.keep.items()})
        self.out = torch.full((8,), float("nan"), dtype=torch.float64, device=dev)
        self.t = t

    def call(self, B, x, y, omega):
        import torch
        xd, yd = self.t(x, torch.float64), self.t(y, torch.float64)
        self.out.fill_(float("nan"))
        stream = torch.cuda.current_stream()
        rc = B.uc_kkt_noalloc(self.lp, xd.data_ptr(), yd.data_ptr(), omega, self.out.data_ptr(),
                              stream.cuda_stream)
        assert rc == B.UC_OK, B.lib.uc_last_error()
        torch.cuda.synchronize()
        return self.out.cpu().numpy().copy()


def oracle_outputs(S, x, y, omega):
    """The eight outputs as the oracle defines them, for a scaled point (x, y)."""
    U = pdhg._unscaled_lp(S)
    rel = kkt.relative_kkt(U, S.Dc * x, S.Dr * y)
    r = kkt.residuals(S.A, S.q, S.c, S.l, S.u, S.m_eq, x, y)
    w = kkt.weighted_kkt(float(r.rp @ r.rp), float(r.rd @ r.rd), r.gap, omega)
    rpu = kkt.residuals(U.A, U.q, U.c, U.l, U.u, U.m_eq, S.Dc * x, S.Dr * y).rp
    return np.array([rel[0], rel[1], rel[2], w, r.pobj, r.dobj, float(np.max(np.abs(rpu), initial=0.0)), 0.0])


def check_against_oracle(got, ref):
    # summation order differs (per-CTA partials, fixed-order tree); ITERATE_RTOL is
    # the tolerance of every FP64 parity test in this suite
    np.testing.assert_allclose(got[:7], ref[:7], rtol=ITERATE_RTOL, atol=0.0)
    assert got[7] == 0.0


def two_calls_in_a_row(B, dlp, x, y, omega):
    import torch
    first = dlp.call(B, x, y, omega)          # the first call on a device may load the kernels
    free0, _ = torch.cuda.mem_get_info()
    second = dlp.call(B, x, y, omega)
    third = dlp.call(B, x, y, omega)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    np.testing.assert_array_equal(second, first)
    np.testing.assert_array_equal(third, first)
    return first


def test_kkt_noalloc_tiny_matches_oracle_and_solver(B):
    P = ucgen.tiny(0)
    raw, ps_o, S = oracle_pipeline(P)
    ps = B.uc_presolve(B.uc_build_lp(P))
    res, rc = B.uc_solve(ps, tol=KKT_TOL)
    assert rc == B.UC_OK
    st = B.uc_get_stats(res)
    n, m, _, _ = B.uc_presolved_dims(ps)
    x, y = B.uc_get_iterate(res, 2, n, m)            # the returned point, scaled presolved LP
    dlp = DeviceLp(B, S)
    got = two_calls_in_a_row(B, dlp, x, y, st["omega"])
    check_against_oracle(got, oracle_outputs(S, x, y, st["omega"]))
    np.testing.assert_allclose(got[:3], [st["rel_primal"], st["rel_dual"], st["rel_gap"]],
                               rtol=ITERATE_RTOL, atol=0.0)
    assert got[6] == pytest.approx(st["abs_primal"], rel=ITERATE_RTOL)
    assert max(got[:3]) <= KKT_TOL


def test_kkt_noalloc_paper_scale_matches_oracle(B):
    P = ucgen.paper_scale(0)
    raw, ps_o, S = oracle_pipeline(P)
    m, n = S.A.shape
    assert -(-m // 1024) + -(-n // 1024) > 4 * 256          # several passes of the finishing loop
    rng = np.random.default_rng(11)
    x = np.clip(rng.standard_normal(n) * 3.0, S.l, S.u)
    y = rng.standard_normal(m)
    y[S.m_eq:] = np.abs(y[S.m_eq:])
    dlp = DeviceLp(B, S)
    for omega in (0.7, 3.0):
        got = two_calls_in_a_row(B, dlp, x, y, omega)
        check_against_oracle(got, oracle_outputs(S, x, y, omega))


def test_kkt_noalloc_propagates_nan(B):
    P = ucgen.tiny(0)
    raw, ps_o, S = oracle_pipeline(P)
    m, n = S.A.shape
    dlp = DeviceLp(B, S)
    x = np.clip(np.zeros(n), S.l, S.u)
    y = np.zeros(m)
    # a column with an entry in an equality row and one in a ">=" row
    A = S.A.tocsc()
    j = next(j for j in range(n)
             if np.any(A.indices[A.indptr[j]:A.indptr[j + 1]] < S.m_eq)
             and np.any(A.indices[A.indptr[j]:A.indptr[j + 1]] >= S.m_eq))
    xn = x.copy()
    xn[j] = np.nan
    got = dlp.call(B, xn, y, 1.0)
    assert np.isnan(got[0]) and np.isnan(got[2]) and np.isnan(got[3]) and np.isnan(got[6])
    assert not np.isnan(got[1])                     # the dual residual does not involve x
    # a NaN only in ">=" rows: min(r, 0) must not drop it
    xi = x.copy()
    jj = next(j for j in range(n) if A.indptr[j + 1] > A.indptr[j]
              and np.all(A.indices[A.indptr[j]:A.indptr[j + 1]] >= S.m_eq))
    xi[jj] = np.nan
    got = dlp.call(B, xi, y, 1.0)
    assert np.isnan(got[0]) and np.isnan(got[6])
    yn = y.copy()
    yn[S.m_eq] = np.nan
    got = dlp.call(B, x, yn, 1.0)
    assert np.isnan(got[1]) and np.isnan(got[2]) and np.isnan(got[3])
    # and a clean point afterwards is unaffected by what the NaN calls left in the scratch
    check_against_oracle(dlp.call(B, x, y, 1.0), oracle_outputs(S, x, y, 1.0))


def test_kkt_noalloc_refuses_sizes_beyond_the_scratch(B):
    import torch
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    xd = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for n, m in ((5_000_000, 4_000_000), (2**31 - 1, 2**31 - 1), (2**31 - 1, 0)):
        big = B.uc_device_lp(n=n, m=m, m_eq=0)
        rc = B.uc_kkt_noalloc(big, xd.data_ptr(), xd.data_ptr(), 1.0, out.data_ptr(), stream)
        assert rc == B.UC_EINVAL and b"too large" in B.lib.uc_last_error(), (n, m)
