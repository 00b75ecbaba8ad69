"""Host side of the C ABI on CPU: the library loads, exports every symbol the
header declares, and its LP builder / presolve / scaling agree with the
oracle's independently written ones."""
import ctypes
import os
import re

import numpy as np
import pytest

import ucgen
from oracle import kkt, lp as olp, presolve as ops

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    import paper_2607_03627_gb300 as pkg
    pkg.build()
    from paper_2607_03627_gb300 import binding
    return binding


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "uc_pdhg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(uc_[a-z_0-9]+)\s*\(", src)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def test_library_exports_every_declared_symbol(B):
    lib = ctypes.CDLL(B.LIB_PATH)
    names = _declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def _problems():
    yield ucgen.tiny(0)
    yield ucgen.make_problem(3, B=25, L=40, G=9, T=7, lo=0.4, hi=0.9, noise=0.05, zero_pmin_frac=0.3)
    P = ucgen.micro(2, B=5, L=6, G=3, T=3)
    P.voll = 0.0                                   # strict balance: no shed columns
    yield P


@pytest.mark.parametrize("P", list(_problems()), ids=lambda P: P.name or "strict")
def test_builder_matches_oracle_exactly(B, P):
    ref = olp.build_lp(P)
    d = B.uc_lp_export(B.uc_build_lp(P))
    assert (d["n"], d["m"], d["m_eq"]) == (ref.n, ref.m, ref.m_eq)
    np.testing.assert_array_equal(d["rowptr"], ref.A.indptr)
    np.testing.assert_array_equal(d["colidx"], ref.A.indices)
    np.testing.assert_array_equal(d["val"], ref.A.data)
    for k in ("q", "c", "l", "u"):
        np.testing.assert_array_equal(d[k], getattr(ref, k))


@pytest.mark.parametrize("aggressive,angles", [(0, 0), (1, 0), (0, 1), (1, 1)],
                         ids=["default", "aggressive", "angles", "angles+aggressive"])
@pytest.mark.parametrize("P", list(_problems()), ids=lambda P: P.name or "strict")
def test_presolve_and_scaling_match_oracle(B, P, aggressive, angles):
    ps_o = ops.presolve(olp.build_lp(P), aggressive=bool(aggressive), angles=bool(angles))
    S = ops.scale(ps_o.lp)
    d = B.uc_presolved_export(B.uc_presolve(B.uc_build_lp(P), aggressive=aggressive, eliminate_angles=angles))
    assert (d["n"], d["m"], d["m_eq"]) == (ps_o.lp.n, ps_o.lp.m, ps_o.lp.m_eq)
    np.testing.assert_array_equal(d["col_map"], ps_o.col_map)
    np.testing.assert_array_equal(d["row_map"], ps_o.row_map)
    np.testing.assert_array_equal(d["rowptr"], S.A.indptr)
    np.testing.assert_array_equal(d["colidx"], S.A.indices)
    np.testing.assert_allclose(d["val"], S.A.data, rtol=1e-13)
    for k, ref in (("q", S.q), ("c", S.c), ("Dr", S.Dr), ("Dc", S.Dc)):
        np.testing.assert_allclose(d[k], ref, rtol=1e-13, err_msg=k)
    for k, ref in (("l", S.l), ("u", S.u)):
        fin = np.isfinite(ref)
        np.testing.assert_array_equal(np.isfinite(d[k]), fin)
        np.testing.assert_allclose(d[k][fin], ref[fin], rtol=1e-13, err_msg=k)
    assert d["eta"] == pytest.approx(S.eta, rel=1e-11)
    assert d["omega0"] == pytest.approx(S.omega0, rel=1e-12)
    assert d["obj_const"] == pytest.approx(ps_o.lp.obj_const, rel=1e-14, abs=1e-9)
    assert d["q_inf"] == S.q_inf_unscaled and d["c_inf"] == S.c_inf_unscaled


@pytest.mark.parametrize("pc", [1, 0], ids=["pock_chambolle", "ruiz_only"])
def test_step_comes_from_a_certified_bound(B, pc):
    # eta = 0.998 / max(U, power estimate), U an upper bound on ||A_s||_2, so that
    # eta ||A_s||_2 < 1 (checked with a dense SVD); the oracle takes the same bound
    P = ucgen.make_problem(7, B=37, L=53, G=11, T=5, lo=0.5, hi=0.9, noise=0.05, zero_pmin_frac=0.2)
    d = B.uc_presolved_export(B.uc_presolve(B.uc_build_lp(P), pock_chambolle=pc))
    S = ops.scale(ops.presolve(olp.build_lp(P)).lp, pock_chambolle=bool(pc))
    A = np.zeros((d["m"], d["n"]))
    for i in range(d["m"]):
        A[i, d["colidx"][d["rowptr"][i]:d["rowptr"][i + 1]]] = d["val"][d["rowptr"][i]:d["rowptr"][i + 1]]
    smax = float(np.linalg.svd(A, compute_uv=False)[0])
    assert d["norm_A"] <= smax * (1 + 1e-12) <= d["norm_bound"] * (1 + 1e-12)
    assert d["eta"] == 0.998 / d["norm_bound"] and d["eta"] * smax < 1.0
    assert d["norm_bound"] == pytest.approx(S.norm_bound, rel=1e-13)
    assert d["eta"] == pytest.approx(S.eta, rel=1e-13)
    if pc:
        assert d["norm_bound"] == 1.0


def test_builder_rejects_bad_data(B):
    P = ucgen.micro(0, B=3, L=3, G=2, T=2)
    bad = P.copy(); bad.line_to = bad.line_from.copy()
    with pytest.raises(B.UCError, match="self loop"):
        B.uc_build_lp(bad)
    bad = P.copy(); bad.x_pu[0] = 0.0
    with pytest.raises(B.UCError, match="reactance"):
        B.uc_build_lp(bad)
    bad = P.copy(); bad.pmin[0] = bad.pmax[0] + 1
    with pytest.raises(B.UCError, match="pmin"):
        B.uc_build_lp(bad)
    bad = P.copy(); bad.load[0, 0] = -1.0
    with pytest.raises(B.UCError, match="load"):
        B.uc_build_lp(bad)
    bad = P.copy(); bad.gen_bus[0] = 99
    with pytest.raises(B.UCError, match="out of range"):
        B.uc_build_lp(bad)


def test_presolve_reports_infeasible(B):
    # strict balance with more load than generation and line capacity can serve
    P = ucgen.micro(0, B=2, L=1, G=1, T=1)
    P.voll = 0.0
    P.load[:] = 0.0
    P.gen_bus[:] = 0
    P.pmax[:] = 0.0
    P.pmin[:] = 0.0
    P.load[0, 0] = 5.0                          # bus 0: only p (fixed 0) and f
    P.fmax[:] = 0.0                             # f fixed at 0 -> balance row empty with rhs 5
    with pytest.raises(B.UCError, match="infeasible"):
        B.uc_presolve(B.uc_build_lp(P))


def test_presolve_does_not_depend_on_the_thread_count(B):
    # large enough that every parallel loop (scaling, power iteration) runs many chunks
    P = ucgen.make_problem(2, B=400, L=530, G=48, T=24, lo=0.5, hi=0.85, noise=0.05, zero_pmin_frac=0.1)
    lp = B.uc_build_lp(P)
    ref = B.uc_presolved_export(B.uc_presolve(lp, threads=1))
    for th in (2, 3, 8):
        d = B.uc_presolved_export(B.uc_presolve(lp, threads=th))
        for k in ("rowptr", "colidx", "val", "q", "c", "l", "u", "Dr", "Dc"):
            np.testing.assert_array_equal(d[k], ref[k], err_msg=f"{k} threads={th}")
        for k in ("eta", "omega0", "norm_A"):
            assert d[k] == ref[k], (k, th)


def test_power_device_option_is_checked(B):
    lp = B.uc_build_lp(ucgen.tiny(0))
    with pytest.raises(B.UCError, match="power_device"):
        B.uc_presolve(lp, power_device=2)
    with pytest.raises(TypeError, match="unknown presolve option"):
        B.uc_presolve(lp, power_devcie=1)


def test_power_device_without_a_device_fails_loudly(B):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(B.UCError, match="no CUDA device"):
        B.uc_presolve(B.uc_build_lp(ucgen.tiny(0)), power_device=1)


def _warp_sectors(rp, ci, order, inv_cols):
    """Distinct 32-byte sectors a warp's gathers touch per gathered FP64 value,
    for rows visited in `order` (device order) gathering at inv_cols[col]."""
    L = np.diff(rp)[order]
    secs = gathers = 0
    for q in range(int(L.max())):
        has = L > q
        rows = order[has]
        warp = np.nonzero(has)[0] // 32
        sector = (inv_cols[ci[rp[rows] + q]] * 8) // 32
        secs += len(np.unique(warp.astype(np.int64) * (1 << 32) + sector))
        gathers += len(rows)
    return secs / gathers


@pytest.mark.parametrize("which", ["tiny", "paper"])
def test_device_order_is_entity_major_and_length_windowed(B, which):
    P = ucgen.tiny(0) if which == "tiny" else ucgen.paper_scale(0)
    ps = B.uc_presolve(B.uc_build_lp(P))
    d = B.uc_presolved_export(ps)
    n, m, m_eq = d["n"], d["m"], d["m_eq"]
    prow, pcol = B.uc_presolved_device_order(ps)
    np.testing.assert_array_equal(np.sort(prow), np.arange(m))
    np.testing.assert_array_equal(np.sort(pcol), np.arange(n))
    assert (prow[:m_eq] < m_eq).all()                    # equality rows keep the first positions
    rp, ci = d["rowptr"].astype(np.int64), d["colidx"].astype(np.int64)
    lr = np.diff(rp)
    lc = np.bincount(ci, minlength=n)
    for order, lens, blocks in ((prow, lr, [(0, m_eq), (m_eq, m)]), (pcol, lc, [(0, n)])):
        for b0, b1 in blocks:
            for w0 in range(b0, b1, 1024):
                w = lens[order[w0:min(b1, w0 + 1024)]]
                assert (np.diff(w) <= 0).all()           # decreasing length inside a window
    nat_r, nat_c = B.uc_presolved_device_order(ps, reorder=False)
    np.testing.assert_array_equal(nat_r, np.arange(m))
    np.testing.assert_array_equal(nat_c, np.arange(n))
    if which == "paper":
        # what the layout is for: a warp's gathers hit few sectors (natural order: ~0.69)
        ATc = np.argsort(ci, kind="stable")
        icol = np.empty(n, np.int64); icol[pcol] = np.arange(n)
        irow = np.empty(m, np.int64); irow[prow] = np.arange(m)
        rows_of = np.repeat(np.arange(m), lr)
        rpT = np.concatenate([[0], np.cumsum(lc)])
        ciT = rows_of[ATc]
        assert _warp_sectors(rp, ci, prow.astype(np.int64), icol) <= 0.3
        assert _warp_sectors(rpT, ciT, pcol.astype(np.int64), irow) <= 0.3
        assert _warp_sectors(rp, ci, np.arange(m), np.arange(n)) >= 0.6


def _c_solve(B, pss, **kw):
    """The C entry point called directly (the Python binding refuses to solve
    without a CUDA device): (status, last error)."""
    import ctypes
    o, keep = B.solve_opts(**kw)
    arr = (ctypes.c_void_p * len(pss))(*[p.ptr for p in pss])
    outs = (ctypes.c_void_p * len(pss))()
    if len(pss) == 1:
        rc = B.lib.uc_solve(pss[0].ptr, ctypes.byref(o), None, outs)
    else:
        rc = B.lib.uc_solve_batch(arr, len(pss), ctypes.byref(o), None, outs)
    return rc, B.lib.uc_last_error().decode()


@pytest.mark.parametrize("kw,msg", [
    (dict(n_eval=3), "n_eval must be even"),
    (dict(max_iter=-1), "max_iter must be"),
    (dict(spmv_kernel=3), "spmv_kernel must be"),
    (dict(stages=1), "stages must be"),
    (dict(cta_rows=100), "cta_rows must be"),
    (dict(rows_per_thread=[3]), "rows_per_thread must be"),
    (dict(adaptive_step=True), "adaptive_step needs"),                  # Halpern
    (dict(algorithm="average", spmv_kernel=2), "staged kernels need"),
    (dict(pw_gains=(-0.5, 0.0, 0.0)), "pw_kp, pw_ki and pw_kd must be"),
    (dict(pw_guard=0.5), "pw_guard must be 0"),
    (dict(pw_guard=float("nan")), "pw_guard must be 0"),
])
def test_solve_rejects_bad_options_before_touching_the_device(B, kw, msg):
    ps = B.uc_presolve(B.uc_build_lp(ucgen.tiny(0)))
    rc, err = _c_solve(B, [ps], **kw)
    assert rc == B.UC_EINVAL and msg in err, (rc, err)


def test_sessions_reject_bad_shapes_before_touching_the_device(B):
    import ctypes
    ps = B.uc_presolve(B.uc_build_lp(ucgen.tiny(0)))
    for pss, kw, msg in (([ps] * 3, dict(lanes=True), "lanes sessions hold 2 or 4"),
                         ([ps] * 2, dict(lanes=True, algorithm="average"), "lanes sessions run the Halpern"),
                         ([ps] * 2, dict(algorithm="average", adaptive_step=True), "adaptive_step needs")):
        rc, err = _c_solve(B, pss, **kw)
        assert rc == B.UC_EINVAL and msg in err, (rc, err)
    out = ctypes.c_void_p()
    assert B.lib.uc_solve(None, None, None, ctypes.byref(out)) == B.UC_EINVAL
    assert b"null argument" in B.lib.uc_last_error()
    assert B.lib.uc_session_create(None, 1, None, None, ctypes.byref(out)) == B.UC_EINVAL


def test_python_solve_fails_loudly_without_a_device(B):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    ps = B.uc_presolve(B.uc_build_lp(ucgen.tiny(0)))
    with pytest.raises(RuntimeError, match="needs a CUDA device"):
        B.uc_solve(ps)


def _device_csr(d, prow, pcol, transpose):
    """The device-order matrix (rows in device order, columns relabelled to device
    positions, each row's entries in their original order), built here."""
    import scipy.sparse as sp
    A = sp.csr_matrix((d["val"], d["colidx"], d["rowptr"]), shape=(d["m"], d["n"]))
    M = A.T.tocsr() if transpose else A
    rorder = (pcol if transpose else prow).astype(np.int64)
    cperm = (prow if transpose else pcol).astype(np.int64)
    cinv = np.empty(len(cperm), np.int64)
    cinv[cperm] = np.arange(len(cperm))
    lens = np.diff(M.indptr)[rorder]
    indptr = np.concatenate([[0], np.cumsum(lens)])
    take = np.concatenate([np.arange(M.indptr[r], M.indptr[r + 1]) for r in rorder]) if len(rorder) else []
    return indptr, cinv[M.indices[take]], M.data[take]


@pytest.mark.parametrize("which", ["tiny", "paper"])
@pytest.mark.parametrize("transpose", [False, True])
def test_strided_groups_describe_the_device_matrix_exactly(B, which, transpose):
    P = ucgen.tiny(0) if which == "tiny" else ucgen.paper_scale(0)
    ps = B.uc_presolve(B.uc_build_lp(P))
    d = B.uc_presolved_export(ps)
    prow, pcol = B.uc_presolved_device_order(ps)
    rp, ci, va = _device_csr(d, prow, pcol, transpose)
    g = B.uc_presolved_strided_groups(ps, transpose)
    G = 16
    rows = len(rp) - 1
    assert g["groups"] == (rows + G - 1) // G and g["entries"] == len(ci)
    rng = np.random.default_rng(0)
    groups = np.arange(g["groups"]) if which == "tiny" else rng.choice(g["groups"], 3000, replace=False)
    for gi in groups:
        r0 = gi * G
        k = int(g["k"][gi])
        o = int(g["off"][gi])
        if k >= 0:
            cols, vals = g["col"][o:o + k], g["val"][o:o + k]
            for s in range(G):
                e0, e1 = rp[r0 + s], rp[r0 + s + 1]
                np.testing.assert_array_equal(ci[e0:e1], cols + s)
                np.testing.assert_array_equal(va[e0:e1], vals)
        elif r0 + G <= rows:    # a full group left on the CSR path really breaks the pattern
            lens = np.diff(rp[r0:r0 + G + 1])
            if lens.min() == lens.max() and lens[0] > 0:
                C = np.stack([ci[rp[r0 + s]:rp[r0 + s + 1]] for s in range(G)])
                V = np.stack([va[rp[r0 + s]:rp[r0 + s + 1]] for s in range(G)])
                assert not ((C - C[0] == np.arange(G)[:, None]).all() and (V == V[0]).all())
    assert int(g["k"][g["k"] >= 0].astype(np.int64).sum()) == g["slots"]
    assert g["strided_entries"] == int((g["k"][g["k"] >= 0].astype(np.int64) * G).sum())
    if which == "paper":   # the time-expanded structure the layout exposes
        assert g["strided_entries"] / g["entries"] >= (0.9 if transpose else 0.85)


@pytest.mark.parametrize("which", ["tiny", "paper"])
def test_presolve_reuse_equals_a_full_presolve_on_the_host(B, which):
    base = ucgen.tiny(3) if which == "tiny" else ucgen.paper_scale(0)
    ps0 = B.uc_presolve(B.uc_build_lp(base))
    Q = ucgen.served_request(base, 1, 7)
    full = B.uc_presolved_export(B.uc_presolve(B.uc_build_lp(Q)))
    re = B.uc_presolved_export(B.uc_presolve_reuse(ps0, B.uc_build_lp(Q)))
    for k in ("rowptr", "colidx", "val", "q", "c", "l", "u", "Dr", "Dc", "col_map", "row_map"):
        np.testing.assert_array_equal(re[k], full[k], err_msg=k)
    for k in ("eta", "omega0", "q_inf", "c_inf", "obj_const"):
        assert re[k] == full[k], k
    with pytest.raises(B.UCError, match="matrix differs"):
        B.uc_presolve_reuse(ps0, B.uc_build_lp(ucgen.tiny(4) if which == "tiny" else ucgen.tiny(0)))


def test_aggressive_postsolve_matches_oracle(B):
    # the host postsolve of a point of the aggressively presolved 30-bus LP (the
    # oracle simplex optimum of that LP) equals the oracle's: substituted shed
    # columns and the duals of the removed doubleton rows included
    from oracle import simplex
    P = ucgen.tiny(0)
    raw = olp.build_lp(P)
    ps_o = ops.presolve(raw, aggressive=True)
    assert any(isinstance(d, ops.Doubleton) for d in ps_o.removed_rows)
    S = ops.scale(ps_o.lp)
    r = simplex.solve_lp(ps_o.lp)
    xo, yo = ops.postsolve(ps_o, r.x, r.y)
    ps = B.uc_presolve(B.uc_build_lp(P), aggressive=1)
    res = B.uc_result_from_point(ps, r.x / S.Dc, r.y / S.Dr)
    xr, yr = B.uc_get_raw_solution(res, raw.n, raw.m)
    np.testing.assert_allclose(xr, xo, rtol=1e-9, atol=1e-9 * np.max(np.abs(xo)))
    np.testing.assert_allclose(yr, yo, rtol=1e-9, atol=1e-9 * np.max(np.abs(yo)))
    assert max(kkt.relative_kkt(raw, xr, yr)) <= 1e-8


@pytest.mark.parametrize("aggressive", [0, 1], ids=["angles", "angles+aggressive"])
def test_angle_postsolve_matches_oracle(B, aggressive):
    # the host postsolve of the oracle simplex optimum of the angle-free 30-bus
    # LP equals the oracle's: angles put back down the tree, tree lines' flow
    # rows given their duals; the pair is KKT-optimal on the LP as built
    from oracle import simplex
    P = ucgen.tiny(0)
    raw = olp.build_lp(P)
    ps_o = ops.presolve(raw, aggressive=bool(aggressive), angles=True)
    S = ops.scale(ps_o.lp)
    r = simplex.solve_lp(ps_o.lp)
    xo, yo = ops.postsolve(ps_o, r.x, r.y)
    ps = B.uc_presolve(B.uc_build_lp(P), aggressive=aggressive, eliminate_angles=1)
    res = B.uc_result_from_point(ps, r.x / S.Dc, r.y / S.Dr)
    xr, yr = B.uc_get_raw_solution(res, raw.n, raw.m)
    np.testing.assert_allclose(xr, xo, rtol=1e-9, atol=1e-9 * np.max(np.abs(xo)))
    np.testing.assert_allclose(yr, yo, rtol=1e-9, atol=1e-9 * np.max(np.abs(yo)))
    assert max(kkt.relative_kkt(raw, xr, yr)) <= 1e-8


def test_angle_elimination_option_is_checked(B):
    with pytest.raises(B.UCError, match="eliminate_angles"):
        B.uc_presolve(B.uc_build_lp(ucgen.tiny(0)), eliminate_angles=2)


def test_angle_elimination_reuse_equals_a_full_presolve(B):
    base = ucgen.tiny(3)
    ps0 = B.uc_presolve(B.uc_build_lp(base), eliminate_angles=1)
    Q = ucgen.served_request(base, 1, 7)
    full = B.uc_presolved_export(B.uc_presolve(B.uc_build_lp(Q), eliminate_angles=1))
    re = B.uc_presolved_export(B.uc_presolve_reuse(ps0, B.uc_build_lp(Q)))
    for k in ("rowptr", "colidx", "val", "q", "c", "l", "u", "Dr", "Dc", "col_map", "row_map"):
        np.testing.assert_array_equal(re[k], full[k], err_msg=k)


def test_device_order_puts_long_columns_last(B):
    # on an angle-free LP the columns with more than 32 entries follow all
    # others (a warp each in the primal kernel), keeping their relative order
    P = ucgen.batch_member(24)
    ps = B.uc_presolve(B.uc_build_lp(P), eliminate_angles=1)
    d = B.uc_presolved_export(ps)
    n = d["n"]
    lc = np.bincount(d["colidx"].astype(np.int64), minlength=n)
    prow, pcol = B.uc_presolved_device_order(ps)
    np.testing.assert_array_equal(np.sort(pcol), np.arange(n))
    longv = lc[pcol] > 32
    k = int(longv.sum())
    assert k > 0 and longv[n - k:].all() and not longv[:n - k].any()
    # the default LP has no such column: its kernels keep the one-thread path
    assert not (np.bincount(B.uc_presolved_export(B.uc_presolve(B.uc_build_lp(P)))["colidx"]) > 32).any()


def test_angle_elimination_with_parallel_lines_matches_oracle(B):
    # a grid with two lines between the same buses (a 2-entry cycle) and a
    # 4-bus ring: the host's angle-free presolve equals the oracle's
    P = ucgen.micro(1, B=4, L=5, G=2, T=3)
    P.ref_bus = 0
    P.line_from = np.array([0, 1, 2, 3, 0], np.int32)
    P.line_to = np.array([1, 2, 3, 0, 1], np.int32)
    P.x_pu = np.array([0.1, 0.2, 0.05, 0.15, 0.3])
    P.fmax = np.full(5, 500.0)
    ps_o = ops.presolve(olp.build_lp(P), angles=True)
    S = ops.scale(ps_o.lp)
    d = B.uc_presolved_export(B.uc_presolve(B.uc_build_lp(P), eliminate_angles=1))
    np.testing.assert_array_equal(d["col_map"], ps_o.col_map)
    np.testing.assert_array_equal(d["row_map"], ps_o.row_map)
    np.testing.assert_array_equal(d["rowptr"], S.A.indptr)
    np.testing.assert_array_equal(d["colidx"], S.A.indices)
    np.testing.assert_allclose(d["val"], S.A.data, rtol=1e-13)
