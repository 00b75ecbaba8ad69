"""The allocation-free KKT entry point (uc_kkt_noalloc) against the solver's
own evaluation.

uc_kkt_noalloc serves callers that must not allocate device memory (graph
capture, pre-reserved memory pools); it keeps its scratch in a fixed array of
the library.  Here the existing entry point uc_solve reports the relative KKT
of its returned point; the new entry point, given that same point and the same
LP in caller-owned device memory, must report the same numbers, on every
call (later calls reuse the scratch earlier ones left behind), and the
device's free memory must not change across two calls in a row after the
first call on the device.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import ucgen
from gpu_common import ITERATE_RTOL, KKT_TOL

pytestmark = pytest.mark.gpu


def test_kkt_noalloc_matches_solver_evaluation():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_03627_gb300 as pkg
    pkg.build()
    from paper_2607_03627_gb300 import binding as B

    P = ucgen.tiny(0)
    ps = B.uc_presolve(B.uc_build_lp(P))
    res, rc = B.uc_solve(ps, tol=KKT_TOL)
    assert rc == B.UC_OK
    st = B.uc_get_stats(res)
    n, m, m_eq, nnz = B.uc_presolved_dims(ps)
    x, y = B.uc_get_iterate(res, 2, n, m)
    d = B.uc_presolved_export(ps)
    A = sp.csr_matrix((d["val"], d["colidx"], d["rowptr"]), shape=(m, n))
    AT = A.T.tocsr()
    AT.sort_indices()

    dev = torch.device("cuda", 0)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    keep = dict(A_rowptr=t(d["rowptr"], torch.int32), A_colidx=t(d["colidx"], torch.int32),
                A_val=t(d["val"], torch.float64), AT_rowptr=t(AT.indptr, torch.int32),
                AT_colidx=t(AT.indices, torch.int32), AT_val=t(AT.data, torch.float64),
                c=t(d["c"], torch.float64), l=t(d["l"], torch.float64), u=t(d["u"], torch.float64),
                Dc=t(d["Dc"], torch.float64), q=t(d["q"], torch.float64), Dr=t(d["Dr"], torch.float64))
    lp = B.uc_device_lp(n=n, m=m, m_eq=m_eq, q_inf=d["q_inf"], c_inf=d["c_inf"],
                        **{k: v.data_ptr() for k, v in keep.items()})
    xd, yd = t(x, torch.float64), t(y, torch.float64)
    out = torch.full((8,), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    results = []

    def call():
        out.fill_(float("nan"))
        rc = B.uc_kkt_noalloc(lp, xd.data_ptr(), yd.data_ptr(), st["omega"], out.data_ptr(),
                              stream.cuda_stream)
        assert rc == B.UC_OK, B.lib.uc_last_error()
        torch.cuda.synchronize()
        results.append(out.cpu().numpy().copy())

    # the first call on a device resolves the scratch address and loads the
    # kernels (the driver may take memory for their code); the two calls in a
    # row after it must not change the free device memory
    call()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        call()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    for o in results:
        np.testing.assert_allclose(o[:3], [st["rel_primal"], st["rel_dual"], st["rel_gap"]],
                                   rtol=ITERATE_RTOL, atol=1e-300)
        assert o[6] == pytest.approx(st["abs_primal"], rel=ITERATE_RTOL)
        assert o[5] + d["obj_const"] == pytest.approx(st["dual_objective"], rel=ITERATE_RTOL)
        assert max(o[:3]) <= KKT_TOL
    np.testing.assert_array_equal(results[0], results[1])
    np.testing.assert_array_equal(results[1], results[2])

    # sizes beyond the fixed scratch are refused before any device work
    big = B.uc_device_lp(n=5_000_000, m=4_000_000, m_eq=0)
    rc = B.uc_kkt_noalloc(big, xd.data_ptr(), yd.data_ptr(), 1.0, out.data_ptr(), stream.cuda_stream)
    assert rc == B.UC_EINVAL and b"too large" in B.lib.uc_last_error()
