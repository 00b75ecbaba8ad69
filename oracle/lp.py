"""O-builder: the multi-period DC unit-commitment LP relaxation, written out.

Test infrastructure only (see ``oracle/__init__``).

The paper solves "the same relaxed problem" with PDHG on the GPU and barrier
on the CPU (Sec. II-C, Alg. 1); its full model is the GO Challenge 3
specification (Sec. II-A), which is not available.  The LP here is the DC
relaxation the benchmark configurations define: commitment u, startup v and
dispatch p per unit and period, bus angles theta, line flows f, and a
load-shed slack s priced at VOLL.  u and v are relaxed to [0, 1].

Layout (time-major).  Columns of period t start at t * nc with
nc = 3G + B + L (+ B when VOLL > 0):
    [p_g (G), u_g (G), v_g (G), theta_b (B), f_l (L), s_b (B)]
Rows: all equality rows first, then all ">=" rows.
    E, per t:  balance_b (B):  sum_{g at b} p_g + s_b - sum_{from=b} f_l + sum_{to=b} f_l = d_bt
               flowdef_l (L):  f_l - (theta_from - theta_to) / x_l = 0
    I, per t:  gen_up_g (G):   Pmax u - p >= 0
               gen_lo_g (G):   p - Pmin u >= 0         (u term omitted when Pmin = 0)
               startup_g (G):  v_t - u_t + u_{t-1} >= 0    (t = 0: v - u >= -u0)
               ramp_up_g (G):  p_{t-1} - p_t >= -R          (t >= 1 only)
               ramp_dn_g (G):  p_t - p_{t-1} >= -R          (t >= 1 only)
Bounds: p in [0, Pmax], u, v in [0, 1], theta free with theta_ref = 0,
f in [-F, F], s in [0, d].  Objective: min sum c p + c_NL u + c_SU v + VOLL s.
Exact zero coefficients are never stored; each row's columns are ascending.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

# column kinds and row kinds (for postsolve / solution split)
COL_P, COL_U, COL_V, COL_TH, COL_F, COL_S = range(6)
ROW_BAL, ROW_FLOW, ROW_GUP, ROW_GLO, ROW_SU, ROW_RUP, ROW_RDN = range(7)


@dataclasses.dataclass
class LP:
    """min c.x  s.t.  A[:m_eq] x = q[:m_eq],  A[m_eq:] x >= q[m_eq:],  l <= x <= u."""
    A: sp.csr_matrix
    q: np.ndarray
    c: np.ndarray
    l: np.ndarray
    u: np.ndarray
    m_eq: int
    obj_const: float = 0.0
    col_kind: np.ndarray | None = None  # int8 per column
    col_t: np.ndarray | None = None     # period per column
    col_idx: np.ndarray | None = None   # unit / bus / line index per column
    row_kind: np.ndarray | None = None
    row_t: np.ndarray | None = None
    row_idx: np.ndarray | None = None

    @property
    def n(self) -> int:
        return self.A.shape[1]

    @property
    def m(self) -> int:
        return self.A.shape[0]


def build_lp(P) -> LP:
    """Build the raw LP of a ``ucgen.UCProblem`` (model as in the module docstring)."""
    B, L, G, T = P.B, P.L, P.G, P.T
    has_s = P.voll > 0.0
    nc = 3 * G + B + L + (B if has_s else 0)
    n = T * nc

    def col_p(t, g): return t * nc + g
    def col_u(t, g): return t * nc + G + g
    def col_v(t, g): return t * nc + 2 * G + g
    def col_th(t, b): return t * nc + 3 * G + b
    def col_f(t, l): return t * nc + 3 * G + B + l
    def col_s(t, b): return t * nc + 3 * G + B + L + b

    # columns: costs and bounds
    c = np.zeros(n)
    lo = np.zeros(n)
    hi = np.zeros(n)
    col_kind = np.zeros(n, np.int8)
    col_t = np.zeros(n, np.int32)
    col_idx = np.zeros(n, np.int32)
    for t in range(T):
        for g in range(G):
            j = col_p(t, g); c[j] = P.c_lin[g]; lo[j] = 0.0; hi[j] = P.pmax[g]
            col_kind[j] = COL_P; col_t[j] = t; col_idx[j] = g
            j = col_u(t, g); c[j] = P.c_nl[g]; lo[j] = 0.0; hi[j] = 1.0
            col_kind[j] = COL_U; col_t[j] = t; col_idx[j] = g
            j = col_v(t, g); c[j] = P.c_su[g]; lo[j] = 0.0; hi[j] = 1.0
            col_kind[j] = COL_V; col_t[j] = t; col_idx[j] = g
        for b in range(B):
            j = col_th(t, b)
            if b == P.ref_bus:
                lo[j] = 0.0; hi[j] = 0.0
            else:
                lo[j] = -np.inf; hi[j] = np.inf
            col_kind[j] = COL_TH; col_t[j] = t; col_idx[j] = b
        for l in range(L):
            j = col_f(t, l); lo[j] = -P.fmax[l]; hi[j] = P.fmax[l]
            col_kind[j] = COL_F; col_t[j] = t; col_idx[j] = l
        if has_s:
            for b in range(B):
                j = col_s(t, b); c[j] = P.voll; lo[j] = 0.0; hi[j] = P.load[t, b]
                col_kind[j] = COL_S; col_t[j] = t; col_idx[j] = b

    rows: list[dict[int, float]] = []
    rhs: list[float] = []
    rkind: list[int] = []
    rt: list[int] = []
    ridx: list[int] = []

    def add(entries: dict[int, float], b: float, kind: int, t: int, idx: int):
        rows.append({j: v for j, v in entries.items() if v != 0.0})
        rhs.append(float(b)); rkind.append(kind); rt.append(t); ridx.append(idx)

    gens_at = [[] for _ in range(B)]
    for g in range(G):
        gens_at[int(P.gen_bus[g])].append(g)
    lines_from = [[] for _ in range(B)]
    lines_to = [[] for _ in range(B)]
    for l in range(L):
        lines_from[int(P.line_from[l])].append(l)
        lines_to[int(P.line_to[l])].append(l)

    # equality rows
    for t in range(T):
        for b in range(B):
            e = {}
            for g in gens_at[b]:
                e[col_p(t, g)] = 1.0
            if has_s:
                e[col_s(t, b)] = 1.0
            for l in lines_from[b]:
                e[col_f(t, l)] = -1.0
            for l in lines_to[b]:
                e[col_f(t, l)] = 1.0
            add(e, P.load[t, b], ROW_BAL, t, b)
        for l in range(L):
            inv_x = 1.0 / P.x_pu[l]
            e = {col_f(t, l): 1.0,
                 col_th(t, int(P.line_from[l])): -inv_x,
                 col_th(t, int(P.line_to[l])): inv_x}
            add(e, 0.0, ROW_FLOW, t, l)
    m_eq = len(rows)
    # inequality rows (>=)
    for t in range(T):
        for g in range(G):
            add({col_u(t, g): P.pmax[g], col_p(t, g): -1.0}, 0.0, ROW_GUP, t, g)
        for g in range(G):
            add({col_p(t, g): 1.0, col_u(t, g): -P.pmin[g]}, 0.0, ROW_GLO, t, g)
        for g in range(G):
            if t == 0:
                add({col_v(t, g): 1.0, col_u(t, g): -1.0}, -P.u0[g], ROW_SU, t, g)
            else:
                add({col_v(t, g): 1.0, col_u(t, g): -1.0, col_u(t - 1, g): 1.0},
                    0.0, ROW_SU, t, g)
        if t >= 1:
            for g in range(G):
                add({col_p(t - 1, g): 1.0, col_p(t, g): -1.0}, -P.ramp[g], ROW_RUP, t, g)
            for g in range(G):
                add({col_p(t, g): 1.0, col_p(t - 1, g): -1.0}, -P.ramp[g], ROW_RDN, t, g)

    m = len(rows)
    indptr = np.zeros(m + 1, np.int64)
    for i, r in enumerate(rows):
        indptr[i + 1] = indptr[i] + len(r)
    indices = np.empty(indptr[-1], np.int64)
    data = np.empty(indptr[-1])
    for i, r in enumerate(rows):
        ks = sorted(r)
        indices[indptr[i]:indptr[i + 1]] = ks
        data[indptr[i]:indptr[i + 1]] = [r[k] for k in ks]
    A = sp.csr_matrix((data, indices, indptr), shape=(m, n))
    return LP(A=A, q=np.asarray(rhs), c=c, l=lo, u=hi, m_eq=m_eq,
              col_kind=col_kind, col_t=col_t, col_idx=col_idx,
              row_kind=np.asarray(rkind, np.int8), row_t=np.asarray(rt, np.int32),
              row_idx=np.asarray(ridx, np.int32))


def split_solution(P, lp: LP, x: np.ndarray, y: np.ndarray | None = None) -> dict:
    """Split a raw-LP primal (and dual) vector into named [T, .] arrays.
    lmp[t, b] is the dual of bus b's balance row in period t ($/MWh)."""
    T, G, B, L = P.T, P.G, P.B, P.L
    out = {k: np.zeros((T, s)) for k, s in
           (("p", G), ("u", G), ("v", G), ("theta", B), ("f", L), ("shed", B))}
    names = {COL_P: "p", COL_U: "u", COL_V: "v", COL_TH: "theta", COL_F: "f", COL_S: "shed"}
    for kind, name in names.items():
        sel = lp.col_kind == kind
        out[name][lp.col_t[sel], lp.col_idx[sel]] = x[sel]
    if y is not None:
        lmp = np.zeros((T, B))
        sel = lp.row_kind == ROW_BAL
        lmp[lp.row_t[sel], lp.row_idx[sel]] = y[sel]
        out["lmp"] = lmp
    return out
