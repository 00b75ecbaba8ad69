"""O3: brute force on micro instances (test infrastructure only).

* ``vertex_enum``: the optimum of a bounded LP is attained at a vertex, i.e. a
  point where the equality rows plus n - m_eq further constraints (">=" rows
  held at equality or variable bounds) are active and linearly independent.
  Every such choice is tried; the best feasible point is the LP optimum.
* ``commitment_enum``: the mixed-integer unit-commitment optimum over all
  u in {0,1}^(G*T), each commitment an LP solved by the simplex (Sec. II-C:
  the relaxation is followed by branch-and-bound over the binaries).
"""
from __future__ import annotations

import itertools

import numpy as np

from . import lp as olp
from . import simplex


def vertex_enum(A, q, c, l, u, m_eq: int, tol: float = 1e-9):
    A = np.asarray(A.todense() if hasattr(A, "todense") else A, dtype=np.float64)
    m, n = A.shape
    cons = []  # (row vector, rhs)
    for i in range(m_eq, m):
        cons.append((A[i], q[i]))
    for j in range(n):
        e = np.zeros(n); e[j] = 1.0
        if np.isfinite(l[j]):
            cons.append((e, l[j]))
        if np.isfinite(u[j]) and u[j] != l[j]:
            cons.append((e, u[j]))
    k = n - m_eq
    best = (np.inf, None)
    AE, qE = A[:m_eq], q[:m_eq]
    for combo in itertools.combinations(range(len(cons)), k):
        M = np.vstack([AE] + [cons[t][0][None, :] for t in combo]) if k > 0 else AE
        r = np.concatenate([qE, [cons[t][1] for t in combo]])
        if np.linalg.matrix_rank(M) < n:
            continue
        x = np.linalg.solve(M, r)
        scale = 1.0 + np.max(np.abs(x))
        if np.any(x < l - tol * scale) or np.any(x > u + tol * scale):
            continue
        res = A @ x - q
        if np.any(np.abs(res[:m_eq]) > tol * scale) or np.any(res[m_eq:] < -tol * scale):
            continue
        obj = float(c @ x)
        if obj < best[0]:
            best = (obj, x)
    return best


def commitment_enum(P):
    """Min over all binary commitments of the UC cost (u fixed, rest an LP)."""
    raw = olp.build_lp(P)
    ucols = np.flatnonzero(raw.col_kind == olp.COL_U)
    best = (np.inf, None)
    for bits in itertools.product((0.0, 1.0), repeat=len(ucols)):
        l = raw.l.copy(); u = raw.u.copy()
        l[ucols] = bits; u[ucols] = bits
        r = simplex.solve(raw.A, raw.q, raw.c, l, u, raw.m_eq)
        if r.status == "optimal" and r.obj < best[0]:
            best = (r.obj, np.array(bits))
    return best
