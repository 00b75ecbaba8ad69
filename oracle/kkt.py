"""KKT residuals of  min c.x  s.t.  A_E x = q_E,  A_I x >= q_I,  l <= x <= u.

Test infrastructure only (see ``oracle/__init__``).

The paper's PDHG stops at a convergence tolerance of 1e-4 with an absolute
feasibility tolerance of 1e-5 (Sec. II-D).  The relative criterion is PDLP's
(Applegate et al. 2021) with eps_abs = eps_rel:

  primal residual  r_p = [A_E x - q_E ;  min(A_I x - q_I, 0)]
  reduced cost     lam = c - A^T y,  lam_proj = projection of lam onto the cone
                   the bounds allow (free if both l and u finite, >= 0 if only l,
                   <= 0 if only u, 0 if neither);  r_d = lam - lam_proj
  dual objective   q.y + sum_j l_j max(lam_proj_j, 0) + u_j min(lam_proj_j, 0)
  relative parts   ||r_p||_inf / (1 + ||q||_inf),  ||r_d||_inf / (1 + ||c||_inf),
                   |c.x - dual| / (1 + |c.x| + |dual|)
  relative KKT     max of the three parts (PDLP's L_INF optimality norm; with
                   the l2 norm a 1e-4 stop left objective gaps above 1e-4 on
                   the 30-bus instances, the infinity norm does not).

The weighted error that drives restarts is
  KKT_w = sqrt(w^2 ||r_p||^2 + ||r_d||^2 / w^2 + (c.x - dual)^2).

Primal infeasibility (Farkas): the LP has no feasible point if some direction
y of the dual problem with c = 0 has y_I >= 0, a reduced cost lam = -A^T y
that the bounds allow (lam_proj = lam) and a positive dual objective
q.y + sum_j l_j max(lam_j, 0) + u_j min(lam_j, 0).  A numerical direction is
accepted when that objective is positive and the largest violation (of
lam = lam_proj and of y_I >= 0, infinity norm) is at most eps times it
(PDLP's primal-infeasibility test, eps = 1e-8).
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Residuals:
    rp: np.ndarray       # primal residual vector (m)
    rd: np.ndarray       # dual residual vector (n)
    lam: np.ndarray      # reduced costs (n)
    lam_proj: np.ndarray
    pobj: float
    dobj: float

    @property
    def gap(self) -> float:
        return self.pobj - self.dobj


def project_reduced_cost(lam: np.ndarray, l: np.ndarray, u: np.ndarray) -> np.ndarray:
    lf = np.isfinite(l)
    uf = np.isfinite(u)
    out = np.zeros_like(lam)
    both = lf & uf
    out[both] = lam[both]
    only_l = lf & ~uf
    out[only_l] = np.maximum(lam[only_l], 0.0)
    only_u = uf & ~lf
    out[only_u] = np.minimum(lam[only_u], 0.0)
    return out


def residuals(A, q, c, l, u, m_eq, x, y) -> Residuals:
    Ax = A @ x
    rp = Ax - q
    rp[m_eq:] = np.minimum(rp[m_eq:], 0.0)
    lam = c - A.T @ y
    lp = project_reduced_cost(lam, l, u)
    rd = lam - lp
    pobj = float(np.dot(c, x))
    bound = 0.0
    lf = np.isfinite(l)
    uf = np.isfinite(u)
    bound += float(np.sum(l[lf] * np.maximum(lp[lf], 0.0)))
    bound += float(np.sum(u[uf] * np.minimum(lp[uf], 0.0)))
    dobj = float(np.dot(q, y)) + bound
    return Residuals(rp=rp, rd=rd, lam=lam, lam_proj=lp, pobj=pobj, dobj=dobj)


def relative_kkt(lp, x, y):
    """(rel_primal, rel_dual, rel_gap) of an LP object with fields A, q, c, l, u, m_eq."""
    r = residuals(lp.A, lp.q, lp.c, lp.l, lp.u, lp.m_eq, x, y)
    rel_p = float(np.max(np.abs(r.rp), initial=0.0)) / (1.0 + float(np.max(np.abs(lp.q), initial=0.0)))
    rel_d = float(np.max(np.abs(r.rd), initial=0.0)) / (1.0 + float(np.max(np.abs(lp.c), initial=0.0)))
    rel_g = abs(r.gap) / (1.0 + abs(r.pobj) + abs(r.dobj))
    return rel_p, rel_d, rel_g


def weighted_kkt(rp_sq: float, rd_sq: float, gap: float, omega: float) -> float:
    return float(np.sqrt(omega * omega * rp_sq + rd_sq / (omega * omega) + gap * gap))


INFEASIBLE_EPS = 1e-8


def farkas_ray(lp, y):
    """(objective, violation) of y as a primal-infeasibility direction of the
    LP object (fields A, q, l, u, m_eq); see the module docstring."""
    lam = -(lp.A.T @ y)
    lp_ = project_reduced_cost(lam, lp.l, lp.u)
    lf = np.isfinite(lp.l)
    uf = np.isfinite(lp.u)
    obj = float(np.dot(lp.q, y))
    obj += float(np.sum(lp.l[lf] * np.maximum(lp_[lf], 0.0)))
    obj += float(np.sum(lp.u[uf] * np.minimum(lp_[uf], 0.0)))
    viol = max(float(np.max(np.abs(lam - lp_), initial=0.0)),
               float(np.max(np.maximum(-y[lp.m_eq:], 0.0), initial=0.0)))
    return obj, viol


def is_infeasibility_certificate(lp, y, eps: float = INFEASIBLE_EPS) -> bool:
    obj, viol = farkas_ray(lp, y)
    return obj > 0.0 and viol <= eps * obj


def abs_primal_inf(lp, x) -> float:
    """Largest absolute violation of a row (|r| for equality rows, max(-r, 0)
    for ">=" rows) or of a bound (Sec. II-D absolute feasibility, reported, not
    gated)."""
    r = lp.A @ x - lp.q
    r[lp.m_eq:] = np.minimum(r[lp.m_eq:], 0.0)
    bv = np.maximum(lp.l - x, 0.0) + np.maximum(x - lp.u, 0.0)
    return float(max(np.max(np.abs(r), initial=0.0), np.max(bv, initial=0.0)))
