"""Pins for the oracle LP builder, presolve, scaling and KKT residuals."""
import numpy as np
import pytest

import ucgen
from oracle import brute, closed, kkt, lp as olp, presolve as ops, simplex


def _sizes(P):
    B, L, G, T = P.B, P.L, P.G, P.T
    n = T * (3 * G + B + L + B)
    m_eq = T * (B + L)
    m = m_eq + T * 3 * G + (T - 1) * 2 * G
    zero_pmin = int(np.count_nonzero(P.pmin == 0.0))
    degree = 0
    nnz = T * (G + B + 2 * L) + T * 3 * L + T * 2 * G + T * (2 * G - zero_pmin) \
        + G * 2 + (T - 1) * G * 3 + (T - 1) * 4 * G
    return n, m, m_eq, nnz


def test_builder_sizes_tiny():
    P = ucgen.tiny(0)
    raw = olp.build_lp(P)
    n, m, m_eq, nnz = _sizes(P)
    assert (raw.n, raw.m, raw.m_eq, raw.A.nnz) == (n, m, m_eq, nnz)
    # columns of every row ascending, no stored zeros
    for i in range(raw.m):
        cols = raw.A.indices[raw.A.indptr[i]:raw.A.indptr[i + 1]]
        assert np.all(np.diff(cols) > 0)
    assert np.all(raw.A.data != 0.0)


@pytest.fixture(scope="module")
def small_solved():
    P = ucgen.micro(3, B=12, L=16, G=4, T=6)
    raw = olp.build_lp(P)
    r = simplex.solve_lp(raw)
    assert r.status == "optimal"
    return P, raw, r


def test_power_balance_sums_to_load(small_solved):
    P, raw, r = small_solved
    sol = olp.split_solution(P, raw, r.x, r.y)
    np.testing.assert_allclose(sol["p"].sum(axis=1) + sol["shed"].sum(axis=1),
                               P.load.sum(axis=1), rtol=1e-10, atol=1e-8)


def test_ptdf_flow_identity(small_solved):
    P, raw, r = small_solved
    sol = olp.split_solution(P, raw, r.x, r.y)
    H = closed.ptdf(P)
    inj = closed.injections(P, sol["p"], sol["shed"])
    for t in range(P.T):
        np.testing.assert_allclose(sol["f"][t], H @ inj[t], rtol=1e-8, atol=1e-7)


def test_line_reversal_symmetry(small_solved):
    P, raw, r = small_solved
    Q = P.copy()
    Q.line_from, Q.line_to = P.line_to.copy(), P.line_from.copy()
    raw2 = olp.build_lp(Q)
    r2 = simplex.solve_lp(raw2)
    assert abs(r2.obj - r.obj) <= 1e-9 * abs(r.obj)
    f1 = olp.split_solution(P, raw, r.x)["f"]
    f2 = olp.split_solution(Q, raw2, r2.x)["f"]
    # flows are unique only where the network fixes them; compare through PTDF
    H1, H2 = closed.ptdf(P), closed.ptdf(Q)
    np.testing.assert_allclose(H2, -H1, atol=1e-10)


def test_kkt_zero_at_simplex_optimum_and_positive_off_it(small_solved):
    P, raw, r = small_solved
    assert max(kkt.relative_kkt(raw, r.x, r.y)) <= 1e-9
    x = r.x.copy()
    j = int(np.flatnonzero(raw.col_kind == olp.COL_P)[0])
    x[j] += 1.0                               # break a balance row
    rp, rd, rg = kkt.relative_kkt(raw, x, r.y)
    assert rp > 1e-4
    y = r.y.copy()
    y[raw.m_eq] = -1.0                        # wrong-signed multiplier of a ">=" row
    rp2, rd2, rg2 = kkt.relative_kkt(raw, r.x, y)
    assert rd2 > 1e-6 or rg2 > 1e-6


def test_kkt_sign_conventions():
    # one ">=" row x0 + x1 >= 1, x >= 0, min x0 + 2 x1: optimum x = (1, 0), y = 1
    import scipy.sparse as sp
    class LP: pass
    lp = LP(); lp.A = sp.csr_matrix(np.array([[1.0, 1.0]])); lp.q = np.array([1.0])
    lp.c = np.array([1.0, 2.0]); lp.l = np.zeros(2); lp.u = np.full(2, np.inf); lp.m_eq = 0
    assert max(kkt.relative_kkt(lp, np.array([1.0, 0.0]), np.array([1.0]))) <= 1e-15
    r = kkt.residuals(lp.A, lp.q, lp.c, lp.l, lp.u, 0, np.array([2.0, 0.0]), np.array([0.0]))
    assert r.rp[0] == 0.0                     # slack rows carry no residual
    r = kkt.residuals(lp.A, lp.q, lp.c, lp.l, lp.u, 0, np.array([0.5, 0.0]), np.array([0.0]))
    assert r.rp[0] == -0.5                    # violated rows do
    r = kkt.residuals(lp.A, lp.q, lp.c, lp.l, lp.u, 0, np.array([1.0, 0.0]), np.array([3.0]))
    assert r.rd[0] == -2.0 and r.rd[1] == -1.0  # lower-bounded columns need lam >= 0


@pytest.mark.parametrize("aggressive", [False, True], ids=["default", "aggressive"])
@pytest.mark.parametrize("seed", range(3))
def test_presolve_preserves_optimum(seed, aggressive):
    P = ucgen.make_problem(seed, B=10, L=13, G=5, T=4, lo=0.4, hi=0.8, noise=0.05,
                           zero_pmin_frac=0.4)
    raw = olp.build_lp(P)
    ps = ops.presolve(raw, aggressive=aggressive)
    # doubleton equations (aggressive presolve): the balance row of a bus with one line and no unit
    # holds that line's flow and the bus's shed column only; the shed column
    # (a column singleton) is solved for, in every period
    deg = np.bincount(np.concatenate([P.line_from, P.line_to]), minlength=P.B)
    units = np.bincount(P.gen_bus, minlength=P.B)
    leaf = np.flatnonzero((deg == 1) & (units == 0))
    dbl = [d for d in ps.removed_rows if isinstance(d, ops.Doubleton)]
    assert len(dbl) == (P.T * len(leaf) if aggressive else 0)
    for d in dbl:
        assert raw.row_kind[d.row] == olp.ROW_BAL and raw.row_idx[d.row] in leaf
        assert raw.col_kind[d.s] == olp.COL_S and raw.col_idx[d.s] == raw.row_idx[d.row]
        assert raw.col_kind[d.f] == olp.COL_F
    assert ps.lp.n == raw.n - P.T - len(dbl)           # theta_ref fixed each period
    n_zero = int(np.count_nonzero(P.pmin == 0.0))
    assert ps.lp.m == raw.m - P.T * n_zero - len(dbl)   # p >= 0 singleton rows
    r_raw = simplex.solve_lp(raw)
    r_red = simplex.solve_lp(ps.lp)
    assert r_raw.status == r_red.status == "optimal"
    assert abs(r_raw.obj - r_red.obj) <= 1e-9 * abs(r_raw.obj)
    xr, yr = ops.postsolve(ps, r_red.x, r_red.y)
    assert max(kkt.relative_kkt(raw, xr, yr)) <= 1e-8


def test_presolve_singleton_tightening_and_recovery():
    # min -x0 + x1 s.t. x0 + x1 = 1 (E), 2 x0 >= 1 (I singleton), x0 <= 3 (I singleton a<0), x in [0, 2]
    import scipy.sparse as sp
    A = sp.csr_matrix(np.array([[1.0, 1.0], [2.0, 0.0], [-1.0, 0.0]]))
    raw = olp.LP(A=A, q=np.array([1.0, 1.0, -3.0]), c=np.array([1.0, -1.0]),
                 l=np.zeros(2), u=np.array([2.0, 2.0]), m_eq=1)
    ps = ops.presolve(raw)
    assert ps.lp.m == 1 and ps.lp.l[0] == 0.5 and ps.lp.u[0] == 2.0
    r = simplex.solve_lp(ps.lp)
    xr, yr = ops.postsolve(ps, r.x, r.y)
    np.testing.assert_allclose(xr, [0.5, 0.5])
    ref = simplex.solve_lp(raw)
    assert abs(r.obj - ref.obj) <= 1e-12
    assert max(kkt.relative_kkt(raw, xr, yr)) <= 1e-12


def test_scaling_preserves_optimum():
    P = ucgen.micro(1, B=8, L=10, G=3, T=4)
    ps = ops.presolve(olp.build_lp(P))
    S = ops.scale(ps.lp)
    r = simplex.solve_lp(ps.lp)
    rs = simplex.solve(S.A, S.q, S.c, S.l, S.u, S.m_eq)
    assert abs(rs.obj + ps.lp.obj_const - r.obj) <= 1e-9 * abs(r.obj)
    # scaled optimum mapped back (x = Dc xs, y = Dr ys) is optimal for the unscaled LP
    assert max(kkt.relative_kkt(ps.lp, S.Dc * rs.x, S.Dr * rs.y)) <= 1e-8


def test_ruiz_equilibrates():
    P = ucgen.tiny(1)
    ps = ops.presolve(olp.build_lp(P))
    S = ops.scale(ps.lp, pock_chambolle=False)
    a = abs(S.A)
    for v in (a.max(axis=1).toarray().ravel(), a.max(axis=0).toarray().ravel()):
        assert v.min() >= 1 - 1e-2 and v.max() <= 1 + 1e-2


def test_power_norm():
    rng = np.random.default_rng(0)
    import scipy.sparse as sp
    M = rng.standard_normal((40, 30))
    M[0] *= 10.0                               # clear spectral gap
    A = sp.csr_matrix(M)
    assert abs(ops.power_norm(A) - np.linalg.norm(M, 2)) <= 1e-8 * np.linalg.norm(M, 2)
    # on the scaled UC matrix: never above the true norm, within 1 %
    ps = ops.presolve(olp.build_lp(ucgen.tiny(0)))
    S = ops.scale(ps.lp)
    true = np.linalg.norm(S.A.toarray(), 2)
    assert S.norm_A <= true * (1 + 1e-12) and S.norm_A >= 0.99 * true
    assert true <= 1.0 + 1e-12                 # Pock-Chambolle alpha=1 bounds ||A_s|| by 1


STEP_CASES = [
    ("tiny", lambda: ucgen.tiny(0)),
    ("ragged37", lambda: ucgen.make_problem(7, B=37, L=53, G=11, T=5, lo=0.5, hi=0.9, noise=0.05,
                                            zero_pmin_frac=0.2)),
    ("micro", lambda: ucgen.micro(2, B=5, L=6, G=3, T=3)),
]


@pytest.mark.parametrize("pc", [True, False], ids=["pock_chambolle", "ruiz_only"])
@pytest.mark.parametrize("name,make", STEP_CASES, ids=[c[0] for c in STEP_CASES])
def test_step_meets_the_pdhg_step_condition(name, make, pc):
    # PDHG converges for tau sigma ||A||^2 = eta^2 ||A_s||^2 < 1: checked with the
    # largest singular value of the dense scaled matrix (LAPACK SVD), which the
    # power estimate approaches from below and the certified bound from above
    S = ops.scale(ops.presolve(olp.build_lp(make())).lp, pock_chambolle=pc)
    smax = float(np.linalg.svd(S.A.toarray(), compute_uv=False)[0])
    assert S.norm_A <= smax * (1 + 1e-12)
    assert S.norm_bound >= smax * (1 - 1e-14)
    assert S.eta * smax < 1.0
    assert S.eta * smax >= 0.998 * (smax / S.norm_bound)
    if pc:
        assert S.norm_bound == 1.0 and smax <= 1.0 + 1e-13


def test_commitment_enumeration_bounds_lp():
    P = ucgen.micro(2, B=2, L=1, G=3, T=3)     # 2^9 commitments
    raw = olp.build_lp(P)
    lp_opt = simplex.solve_lp(raw)
    mip_opt, bits = brute.commitment_enum(P)
    assert mip_opt >= lp_opt.obj - 1e-7 * abs(lp_opt.obj)


def test_commitment_enumeration_equals_lp_when_integral():
    # demand above total capacity: every unit fully on, u* = 1 is integral
    P = ucgen.micro(4, B=2, L=1, G=2, T=2)
    P.load[:] = P.pmax.sum()                   # each bus asks for the full capacity
    raw = olp.build_lp(P)
    r = simplex.solve_lp(raw)
    sol = olp.split_solution(P, raw, r.x)
    assert np.allclose(sol["u"], np.round(sol["u"]), atol=1e-9)
    mip_opt, _ = brute.commitment_enum(P)
    assert abs(mip_opt - r.obj) <= 1e-9 * abs(r.obj)


def test_aggressive_presolve_on_the_30_bus_lp():
    # doubleton equations at every leaf bus without units; the reduced LP has the
    # raw optimum, and postsolve recovers primal and dual points that are
    # KKT-optimal on the raw LP (the recovered rows' duals included)
    P = ucgen.tiny(0)
    raw = olp.build_lp(P)
    base = ops.presolve(raw)
    ps = ops.presolve(raw, aggressive=True)
    dbl = [d for d in ps.removed_rows if isinstance(d, ops.Doubleton)]
    assert len(dbl) > 0 and ps.lp.n == base.lp.n - len(dbl) and ps.lp.m == base.lp.m - len(dbl)
    r_raw = simplex.solve_lp(raw)
    r_red = simplex.solve_lp(ps.lp)
    assert abs(r_raw.obj - r_red.obj) <= 1e-9 * abs(r_raw.obj)
    xr, yr = ops.postsolve(ps, r_red.x, r_red.y)
    assert max(kkt.relative_kkt(raw, xr, yr)) <= 1e-8
    assert abs(float(raw.c @ xr) - r_raw.obj) <= 1e-9 * abs(r_raw.obj)
