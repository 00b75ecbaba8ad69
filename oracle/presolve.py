"""Presolve, diagonal scaling, ||A||_2 estimate and postsolve, written plainly.

Test infrastructure only (see ``oracle/__init__``).

The paper's presolve is Gurobi's (Sec. II-D: fewer rows/columns before the
relaxation); this is the reduced form the GPU arm needs, applied identically
to every load so that the reduced structure does not depend on the load:

  repeat until a pass changes nothing:
    1. every active column with l == u is fixed: its value moves into the row
       right-hand sides and the objective constant;
    2. rows are swept in order, counting entries in active columns:
         0 entries: equality needs q == 0, ">=" needs q <= 0 (else infeasible);
                    the row is dropped;
         1 entry a x_j:  equality fixes l_j = u_j = q / a;  ">=" tightens
                    l_j (a > 0) or u_j (a < 0) to q / a; the row is dropped;
    3. (aggressive presolve only) doubleton equations: equality rows are swept in order; a row with two
       entries a_f x_f + a_s x_s = q in active columns, one of which (x_s) has
       no other entry in an active row, is solved for x_s (when both qualify,
       x_s is the one with the larger index).  x_s's bounds become bounds on
       x_f -- x_f = (q - a_s x_s) / a_f for x_s in [l_s, u_s] -- intersected
       with x_f's own, x_s's cost moves to x_f (c_f -= c_s a_f / a_s, constant
       c_s q / a_s), and the row and x_s leave the LP;
    4. every active column with no entry in an active row is fixed at the bound
       its cost prefers (l if c > 0, u if c < 0, else l, u or 0 when finite).
  Surviving rows and columns keep their original order.

Scaling (the PDLP preconditioner, Applegate et al. 2021): 10 Ruiz passes
(divide row i by sqrt(max_j |a_ij|) and column j by sqrt(max_i |a_ij|), both
taken from the matrix at the start of the pass), then one Pock-Chambolle pass
with alpha = 1 (divide by sqrt of row / column absolute sums).  With the
accumulated factors D_r, D_c:  A_s = D_r A D_c,  c_s = D_c c,  q_s = D_r q,
l_s = l / D_c,  u_s = u / D_c.

||A_s||_2 estimate: power iteration on A_s^T A_s started at 1/sqrt(n), stopped
when the estimate changes by at most 1e-10 relative or after 500 products.

Step size: eta = 0.998 / max(U, estimate), U a certified upper bound on
||A_s||_2.  PDHG converges for tau sigma ||A||^2 < 1, and a power estimate
approaches ||A_s||_2 from below, so the estimate alone can overshoot the step.
After the Pock-Chambolle pass (alpha = 1) the Schur test, with weights the
square roots of the row and column absolute sums the pass divided by, gives
||A_s||_2 <= 1, so U = 1; without that pass U = sqrt(||A_s||_1 ||A_s||_inf)
(the Schur test with unit weights).  Initial primal weight
omega0 = ||c_s|| / ||q_s|| when both exceed 1e-10, else 1.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

from .lp import COL_F, COL_TH, LP, ROW_FLOW

RUIZ_ITERS = 10
PC_ALPHA = 1.0
POWER_TOL = 1e-10
POWER_MAX = 500
ETA_FACTOR = 0.998


class Infeasible(Exception):
    pass


@dataclasses.dataclass
class Presolved:
    lp: LP                    # reduced, unscaled
    col_map: np.ndarray       # reduced column -> raw column
    row_map: np.ndarray       # reduced row -> raw row
    raw_n: int
    raw_m: int
    fixed: list               # (raw col, value) in the order fixed
    removed_rows: list        # (raw row, raw col or -1, coef, kind 'E'/'I', tightened) or a Doubleton
    raw: LP


@dataclasses.dataclass
class Doubleton:
    """A doubleton equation a_f x_f + a_s x_s = q removed by solving for x_s."""
    row: int
    s: int
    a_s: float
    f: int
    a_f: float
    q: float
    lo_from_s: bool           # x_f's lower bound came from x_s's bounds
    hi_from_s: bool           # x_f's upper bound came from x_s's bounds


@dataclasses.dataclass
class AngleElimination:
    """The LP with the bus angles substituted out along a spanning tree (see
    eliminate_angles), and what restore_angles needs to put them back."""
    lp: LP                    # raw columns but the angles, raw rows but the tree lines' flow rows
    col_keep: np.ndarray      # its column -> raw column
    row_keep: np.ndarray      # its row -> raw row
    roots: list               # per period: the reference bus's angle column
    tree: list                # per period, in breadth-first order: (angle col, parent's angle col,
                              #   flow col of the tree line, s, 1/x of the line)
    tree_row_of: dict         # flow col of a tree line -> its (removed) raw flow row


def eliminate_angles(raw: LP) -> AngleElimination:
    """Substitute the free bus angles out of the raw UC LP (Sec. II-A's DC
    network; the paper's aggressive presolve substitutes free columns, Sec.
    II-D).  Per period, the flow-definition rows f_l - inv_l (theta_a - theta_b)
    = 0 (a = from bus, b = to bus, inv_l = 1/x_l) define a graph on the angle
    columns.  A breadth-first spanning tree is grown from the reference bus
    (the angle column fixed at 0), visiting each bus's lines in row order.  A
    tree line's flow row gives theta_child - theta_parent = s f_e / inv_e (s = +1
    when the child is the line's from end, else -1), so every angle difference
    is a sum of tree flows along the tree path.  The tree lines' rows and all
    angle columns leave the LP, and the row of every other line becomes
      f_l - inv_l (sum_{e on a's path up} s_e f_e / inv_e
                   - sum_{e on b's path up} s_e f_e / inv_e) = 0,
    the two paths cut at their common part (Kirchhoff's voltage law on the
    line's fundamental cycle).  The LP is equivalent; the other rows have no
    angle entry."""
    A = raw.A.tocsr()
    th = raw.col_kind == COL_TH
    flow_rows = np.flatnonzero(raw.row_kind == ROW_FLOW)
    new_rows = {}
    drop = set()
    roots, tree, tree_row_of = [], [], {}
    for t in sorted(set(int(v) for v in raw.col_t[th])):
        nodes = [int(j) for j in np.flatnonzero(th & (raw.col_t == t))]
        fixed0 = [j for j in nodes if raw.l[j] == 0.0 and raw.u[j] == 0.0]
        if len(fixed0) != 1:
            raise ValueError(f"period {t}: expected one reference angle, found {len(fixed0)}")
        root = fixed0[0]
        edges = []            # (row, flow col, from angle col, to angle col, inv)
        for i in flow_rows[raw.row_t[flow_rows] == t]:
            fc = a = b = None
            inv = 0.0
            for k in range(A.indptr[i], A.indptr[i + 1]):
                j, v = int(A.indices[k]), float(A.data[k])
                if raw.col_kind[j] == COL_F:
                    fc = j
                elif v < 0:
                    a = j
                else:
                    b, inv = j, v
            edges.append((int(i), fc, a, b, inv))
        adj = {j: [] for j in nodes}
        for e, (_, _, a, b, _) in enumerate(edges):
            adj[a].append((b, e))
            adj[b].append((a, e))
        parent = {root: None}
        order = [root]
        for v in order:                          # breadth-first: order grows while read
            for w, e in adj[v]:
                if w not in parent:
                    parent[w] = (v, e)
                    order.append(w)
        if len(order) != len(nodes):
            raise ValueError(f"period {t}: the grid is not connected")

        def up(v):
            path = []
            while parent[v] is not None:
                p_, e = parent[v]
                path.append((e, 1.0 if edges[e][2] == v else -1.0))
                v = p_
            return path

        in_tree = {parent[w][1] for w in order[1:]}
        for e, (i, fc, a, b, inv) in enumerate(edges):
            if e in in_tree:
                drop.add(i)
                tree_row_of[fc] = i
                continue
            pa, pb = up(a), up(b)
            while pa and pb and pa[-1] == pb[-1]:
                pa.pop()
                pb.pop()
            row = {fc: 1.0}
            for g, sg in pa:
                row[edges[g][1]] = -sg * inv / edges[g][4]
            for g, sg in pb:
                row[edges[g][1]] = sg * inv / edges[g][4]
            new_rows[int(i)] = row
        roots.append(root)
        tree.append([(w, parent[w][0], edges[parent[w][1]][1], 1.0 if edges[parent[w][1]][2] == w else -1.0,
                      edges[parent[w][1]][4]) for w in order[1:]])
    col_keep = np.flatnonzero(~th)
    newcol = -np.ones(raw.n, np.int64)
    newcol[col_keep] = np.arange(col_keep.size)
    row_keep = np.array([i for i in range(raw.m) if i not in drop], np.int64)
    indptr, indices, data = [0], [], []
    for i in row_keep:
        if i in new_rows:
            ents = new_rows[i]
        else:
            ents = {int(A.indices[k]): float(A.data[k]) for k in range(A.indptr[i], A.indptr[i + 1])}
        row = sorted((int(newcol[j]), v) for j, v in ents.items())
        if any(j < 0 for j, _ in row):
            raise ValueError(f"row {i} has an angle entry but is no flow row")
        indices += [j for j, _ in row]
        data += [v for _, v in row]
        indptr.append(len(indices))
    At = sp.csr_matrix((np.array(data, float), np.array(indices, np.int64), np.array(indptr, np.int64)),
                       shape=(row_keep.size, col_keep.size))
    lp = LP(A=At, q=raw.q[row_keep].copy(), c=raw.c[col_keep].copy(), l=raw.l[col_keep].copy(),
            u=raw.u[col_keep].copy(), m_eq=int(np.count_nonzero(row_keep < raw.m_eq)), obj_const=raw.obj_const,
            col_kind=raw.col_kind[col_keep], col_t=raw.col_t[col_keep], col_idx=raw.col_idx[col_keep],
            row_kind=raw.row_kind[row_keep], row_t=raw.row_t[row_keep], row_idx=raw.row_idx[row_keep])
    return AngleElimination(lp=lp, col_keep=col_keep, row_keep=row_keep, roots=roots, tree=tree,
                            tree_row_of=tree_row_of)


def restore_angles(E: AngleElimination, raw: LP, x: np.ndarray, y: np.ndarray | None = None):
    """Map a point of E.lp to the raw LP: the angles from the reference bus's
    value down the tree, theta_child = theta_parent + s f_e / inv_e; the dual
    of a tree line's flow row from the reduced cost of its flow column, which
    the substitution moved into the rows it entered: y_e = sum over the
    substituted rows r holding f_e of (coefficient) * y_r."""
    xr = np.zeros(raw.n)
    xr[E.col_keep] = x
    for root, tr in zip(E.roots, E.tree):
        xr[root] = raw.l[root]
        for w, p_, fc, sg, inv in tr:
            xr[w] = xr[p_] + sg * xr[fc] / inv
    if y is None:
        return xr, None
    yr = np.zeros(raw.m)
    yr[E.row_keep] = y
    A = E.lp.A.tocsr()
    for r in range(A.shape[0]):
        if E.lp.row_kind[r] != ROW_FLOW:
            continue
        for k in range(A.indptr[r], A.indptr[r + 1]):
            fc = int(E.col_keep[A.indices[k]])
            if fc in E.tree_row_of:
                yr[E.tree_row_of[fc]] += A.data[k] * y[r]
    return xr, yr


def presolve(raw: LP, aggressive: bool = False, angles: bool = False) -> Presolved:
    """The reductions of the module docstring; with ``angles`` the bus angles
    are first substituted out (eliminate_angles), and the returned maps still
    point at raw columns and rows (``fixed`` and ``removed_rows`` then refer to
    the angle-free LP)."""
    if not angles:
        return _reduce(raw, aggressive)
    E = eliminate_angles(raw)
    inner = _reduce(E.lp, aggressive)
    ps = Presolved(lp=inner.lp, col_map=E.col_keep[inner.col_map], row_map=E.row_keep[inner.row_map],
                   raw_n=raw.n, raw_m=raw.m, fixed=inner.fixed, removed_rows=inner.removed_rows, raw=raw)
    ps._inner = inner
    ps._angles = E
    return ps


def _reduce(raw: LP, aggressive: bool = False) -> Presolved:
    A = raw.A.tocsr()
    n, m = raw.n, raw.m
    l = raw.l.copy()
    u = raw.u.copy()
    q = raw.q.copy()
    obj_const = raw.obj_const
    col_on = np.ones(n, bool)
    row_on = np.ones(m, bool)
    fixed = []
    removed = []
    xfix = np.zeros(n)
    c = raw.c.copy()
    Acsc = A.tocsc()

    changed = True
    while changed:
        changed = False
        # 1. fixed columns
        for j in range(n):
            if col_on[j] and l[j] == u[j]:
                v = l[j]
                for k in range(Acsc.indptr[j], Acsc.indptr[j + 1]):
                    i = Acsc.indices[k]
                    if row_on[i]:
                        q[i] -= Acsc.data[k] * v
                obj_const += c[j] * v
                xfix[j] = v
                col_on[j] = False
                fixed.append((j, v))
                changed = True
        # 2. empty and singleton rows
        for i in range(m):
            if not row_on[i]:
                continue
            ents = [(A.indices[k], A.data[k]) for k in range(A.indptr[i], A.indptr[i + 1])
                    if col_on[A.indices[k]]]
            is_eq = i < raw.m_eq
            if len(ents) == 0:
                if (is_eq and abs(q[i]) > 1e-9) or ((not is_eq) and q[i] > 1e-9):
                    raise Infeasible(f"empty row {i} with rhs {q[i]}")
                row_on[i] = False
                removed.append((i, -1, 0.0, "E" if is_eq else "I", False))
                changed = True
            elif len(ents) == 1:
                j, a = ents[0]
                bnd = q[i] / a
                tightened = False
                if is_eq:
                    if bnd < l[j] - 1e-9 or bnd > u[j] + 1e-9:
                        raise Infeasible(f"singleton equality row {i}")
                    l[j] = bnd
                    u[j] = bnd
                    tightened = True
                elif a > 0:
                    if bnd > l[j]:
                        l[j] = bnd
                        tightened = True
                else:
                    if bnd < u[j]:
                        u[j] = bnd
                        tightened = True
                if l[j] > u[j] + 1e-9:
                    raise Infeasible(f"bounds crossed on column {j}")
                if l[j] > u[j]:
                    u[j] = l[j]
                row_on[i] = False
                removed.append((i, j, a, "E" if is_eq else "I", tightened))
                changed = True
        # 3. doubleton equations with a column singleton
        def active_entries(j):
            return sum(1 for k in range(Acsc.indptr[j], Acsc.indptr[j + 1]) if row_on[Acsc.indices[k]])
        for i in range(raw.m_eq if aggressive else 0):
            if not row_on[i]:
                continue
            ents = [(A.indices[k], A.data[k]) for k in range(A.indptr[i], A.indptr[i + 1])
                    if col_on[A.indices[k]]]
            if len(ents) != 2:
                continue
            (j1, a1), (j2, a2) = ents
            single = [jj for jj in (j1, j2) if active_entries(jj) == 1]
            if not single:
                continue
            js = max(single)
            (jf, af), (_, a_s) = ((j1, a1), (j2, a2)) if js == j2 else ((j2, a2), (j1, a1))
            v1 = (q[i] - a_s * l[js]) / af
            v2 = (q[i] - a_s * u[js]) / af
            lo, hi = min(v1, v2), max(v1, v2)
            lo_from = bool(lo > l[jf])
            hi_from = bool(hi < u[jf])
            if lo_from:
                l[jf] = lo
            if hi_from:
                u[jf] = hi
            if l[jf] > u[jf] + 1e-9:
                raise Infeasible(f"doubleton row {i}: bounds of column {jf} cross")
            if l[jf] > u[jf]:
                u[jf] = l[jf]
            c[jf] = c[jf] - c[js] * af / a_s
            obj_const += c[js] * q[i] / a_s
            row_on[i] = False
            col_on[js] = False
            removed.append(Doubleton(row=i, s=js, a_s=a_s, f=jf, a_f=af, q=q[i],
                                     lo_from_s=lo_from, hi_from_s=hi_from))
            changed = True
        # 4. empty columns
        for j in range(n):
            if not col_on[j]:
                continue
            used = False
            for k in range(Acsc.indptr[j], Acsc.indptr[j + 1]):
                if row_on[Acsc.indices[k]]:
                    used = True
                    break
            if used:
                continue
            cj = c[j]
            if cj > 0:
                v = l[j]
            elif cj < 0:
                v = u[j]
            else:
                v = l[j] if np.isfinite(l[j]) else (u[j] if np.isfinite(u[j]) else 0.0)
            if not np.isfinite(v):
                raise Infeasible(f"unbounded empty column {j}")
            obj_const += cj * v
            xfix[j] = v
            col_on[j] = False
            fixed.append((j, v))
            changed = True

    col_map = np.flatnonzero(col_on)
    row_map = np.flatnonzero(row_on)
    Ared = A[row_map][:, col_map].tocsr()
    Ared.sort_indices()
    m_eq = int(np.count_nonzero(row_map < raw.m_eq))
    red = LP(A=Ared, q=q[row_map].copy(), c=c[col_map].copy(),
             l=l[col_map].copy(), u=u[col_map].copy(), m_eq=m_eq, obj_const=obj_const)
    ps = Presolved(lp=red, col_map=col_map, row_map=row_map, raw_n=n, raw_m=m,
                   fixed=fixed, removed_rows=removed, raw=raw)
    ps._xfix = xfix
    ps._tight_l = l
    ps._tight_u = u
    return ps


def postsolve(ps: Presolved, x: np.ndarray, y: np.ndarray | None = None):
    """Map a reduced (unscaled) primal/dual pair back to the raw LP.

    Primal: fixed columns take their fixed value.  Dual: removed rows get 0,
    except a singleton row whose bound is active in the reduced solution and
    was tightened by that row: it takes the column's reduced cost / a.
    """
    E = getattr(ps, "_angles", None)
    if E is not None:
        xt, yt = postsolve(ps._inner, x, y)
        return restore_angles(E, ps.raw, xt, yt)
    raw = ps.raw
    xr = ps._xfix.copy()
    xr[ps.col_map] = x
    for d in reversed(ps.removed_rows):          # substituted columns, last removed first
        if isinstance(d, Doubleton):
            xr[d.s] = (d.q - d.a_f * xr[d.f]) / d.a_s
    if y is None:
        return xr, None
    yr = np.zeros(ps.raw_m)
    yr[ps.row_map] = y
    # reduced costs in the raw LP with the rows known so far
    lam = raw.c - raw.A.T @ yr
    for entry in reversed(ps.removed_rows):
        if isinstance(entry, Doubleton):
            d = entry
            # x_f at a bound that came from x_s's bounds: the row's dual makes
            # x_f's reduced cost zero (x_s then sits at its bound); otherwise it
            # makes x_s's zero
            on_lo = d.lo_from_s and abs(xr[d.f] - ps._tight_l[d.f]) <= 1e-9 * (1 + abs(xr[d.f]))
            on_hi = d.hi_from_s and abs(xr[d.f] - ps._tight_u[d.f]) <= 1e-9 * (1 + abs(xr[d.f]))
            if on_lo or on_hi:
                yr[d.row] = (lam[d.f] + d.a_f * yr[d.row]) / d.a_f
            else:
                yr[d.row] = (lam[d.s] + d.a_s * yr[d.row]) / d.a_s
            lam = raw.c - raw.A.T @ yr
            continue
        (i, j, a, kind, tightened) = entry
        if j < 0 or not tightened:
            continue
        if kind == "E":
            yr[i] = lam[j] / a
        else:
            at_bound = abs(xr[j] - (ps._tight_l[j] if a > 0 else ps._tight_u[j])) <= 1e-9 * (1 + abs(xr[j]))
            if at_bound and lam[j] / a > 0:
                yr[i] = lam[j] / a
        lam = raw.c - raw.A.T @ yr
    return xr, yr


@dataclasses.dataclass
class Scaled:
    A: sp.csr_matrix
    q: np.ndarray
    c: np.ndarray
    l: np.ndarray
    u: np.ndarray
    m_eq: int
    Dr: np.ndarray
    Dc: np.ndarray
    eta: float
    omega0: float
    norm_A: float             # power-iteration estimate of ||A_s||_2
    norm_bound: float         # max(U, norm_A): the step is ETA_FACTOR / norm_bound
    q_inf_unscaled: float
    c_inf_unscaled: float


def _row_absmax(A):
    """max_j |a_ij| per row (0 for an empty row)."""
    out = np.zeros(A.shape[0])
    nz = np.diff(A.indptr) > 0
    if A.data.size:
        red = np.maximum.reduceat(np.abs(A.data), A.indptr[:-1][nz])
        out[nz] = red
    return out


def _scale_matrix(A: sp.csr_matrix, rf: np.ndarray, cf: np.ndarray) -> sp.csr_matrix:
    """A_ij / rf_i / cf_j."""
    B = A.copy()
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    B.data = B.data / rf[rows] / cf[B.indices]
    return B


def ruiz_pass(A: sp.csr_matrix):
    absA = abs(A)
    rmax = _row_absmax(absA)
    cmax = _row_absmax(absA.T.tocsr())
    rf = np.where(rmax > 0, np.sqrt(rmax), 1.0)
    cf = np.where(cmax > 0, np.sqrt(cmax), 1.0)
    return _scale_matrix(A, rf, cf), rf, cf


def pock_chambolle_pass(A: sp.csr_matrix, alpha: float = PC_ALPHA):
    absA = abs(A)
    rs = np.asarray((absA.power(2.0 - alpha)).sum(axis=1)).ravel()
    cs = np.asarray((absA.power(alpha)).sum(axis=0)).ravel()
    rf = np.where(rs > 0, np.sqrt(rs), 1.0)
    cf = np.where(cs > 0, np.sqrt(cs), 1.0)
    return _scale_matrix(A, rf, cf), rf, cf


def power_norm(A: sp.csr_matrix, tol: float = POWER_TOL, max_iter: int = POWER_MAX) -> float:
    """||A||_2 by power iteration on A^T A (start 1/sqrt(n))."""
    n = A.shape[1]
    v = np.full(n, 1.0 / np.sqrt(n))
    AT = A.T.tocsr()
    lam_prev = 0.0
    lam = 0.0
    for _ in range(max_iter):
        w = AT @ (A @ v)
        lam = float(np.sqrt(np.dot(w, w)))
        if lam == 0.0:
            return 0.0
        v = w / lam
        if abs(lam - lam_prev) <= tol * lam:
            break
        lam_prev = lam
    return float(np.sqrt(lam))


def norm_upper_bound(A: sp.csr_matrix, pock_chambolle: bool) -> float:
    """Certified upper bound U on ||A||_2 of the scaled matrix (see the module
    docstring): 1 after a Pock-Chambolle pass with alpha = 1, else
    sqrt(max column absolute sum * max row absolute sum)."""
    if pock_chambolle:
        return 1.0
    absA = abs(A)
    r = float(np.max(np.asarray(absA.sum(axis=1)).ravel(), initial=0.0))
    c = float(np.max(np.asarray(absA.sum(axis=0)).ravel(), initial=0.0))
    return float(np.sqrt(r * c))


def scale(lp: LP, ruiz_iters: int = RUIZ_ITERS, pock_chambolle: bool = True) -> Scaled:
    A = lp.A.tocsr().astype(np.float64)
    Dr = np.ones(lp.m)
    Dc = np.ones(lp.n)
    for _ in range(ruiz_iters):
        A, rf, cf = ruiz_pass(A)
        Dr = Dr / rf
        Dc = Dc / cf
    if pock_chambolle:
        A, rf, cf = pock_chambolle_pass(A)
        Dr = Dr / rf
        Dc = Dc / cf
    c = Dc * lp.c
    q = Dr * lp.q
    with np.errstate(invalid="ignore"):
        l = lp.l / Dc
        u = lp.u / Dc
    nrm = power_norm(A)
    bound = max(norm_upper_bound(A, pock_chambolle), nrm)
    eta = ETA_FACTOR / bound if bound > 0 else 1.0
    cn = float(np.linalg.norm(c))
    qn = float(np.linalg.norm(q))
    omega0 = cn / qn if (cn > 1e-10 and qn > 1e-10) else 1.0
    return Scaled(A=A, q=q, c=c, l=l, u=u, m_eq=lp.m_eq, Dr=Dr, Dc=Dc, eta=eta,
                  omega0=omega0, norm_A=nrm, norm_bound=bound,
                  q_inf_unscaled=float(np.max(np.abs(lp.q), initial=0.0)),
                  c_inf_unscaled=float(np.max(np.abs(lp.c), initial=0.0)))
