"""Vertex test of an LP point, written plainly.

Test infrastructure only (see ``oracle/__init__``).

A point x of {A_E x = q_E, A_I x >= q_I, l <= x <= u} is a vertex (basic
feasible solution) exactly when it is feasible and the constraints active at
it -- all equality rows, the ">=" rows it meets with equality and the bounds
it sits on -- contain n linearly independent ones, i.e. the active constraint
matrix has rank n (the number of columns).  This is the definition of a basic
solution; the crossover that follows PDHG in the paper's GPU arm (Sec. II-C,
Alg. 1 "Solver 1") must end at one.
"""
from __future__ import annotations

import numpy as np


def active_matrix(lp, x, tol: float = 1e-9) -> np.ndarray:
    """Dense rows of the constraints active at x (tolerance relative to 1 + |value|)."""
    A = lp.A.toarray()
    n = A.shape[1]
    rows = [A[i] for i in range(lp.m_eq)]
    act = A @ x
    for i in range(lp.m_eq, A.shape[0]):
        if abs(act[i] - lp.q[i]) <= tol * (1.0 + abs(lp.q[i])):
            rows.append(A[i])
    eye = np.eye(n)
    for j in range(n):
        on_l = np.isfinite(lp.l[j]) and abs(x[j] - lp.l[j]) <= tol * (1.0 + abs(lp.l[j]))
        on_u = np.isfinite(lp.u[j]) and abs(x[j] - lp.u[j]) <= tol * (1.0 + abs(lp.u[j]))
        if on_l or on_u:
            rows.append(eye[j])
    return np.array(rows) if rows else np.zeros((0, n))


def is_vertex(lp, x, tol: float = 1e-9) -> bool:
    """Feasible within tol and the active constraints have rank n."""
    r = lp.A @ x - lp.q
    feas = (np.all(np.abs(r[:lp.m_eq]) <= tol * (1.0 + np.abs(lp.q[:lp.m_eq])))
            and np.all(r[lp.m_eq:] >= -tol * (1.0 + np.abs(lp.q[lp.m_eq:])))
            and np.all(x >= lp.l - tol * (1.0 + np.abs(np.nan_to_num(lp.l, posinf=0, neginf=0))))
            and np.all(x <= lp.u + tol * (1.0 + np.abs(np.nan_to_num(lp.u, posinf=0, neginf=0)))))
    if not feas:
        return False
    M = active_matrix(lp, x, tol)
    return M.shape[0] >= lp.A.shape[1] and np.linalg.matrix_rank(M) == lp.A.shape[1]
