"""O4: closed forms and physical invariants of the DC unit-commitment LP.

Test infrastructure only (see ``oracle/__init__``).

* ``merit_order``: one bus, one period, units initially off.  With u relaxed,
  the cheapest way to produce p from unit g sets u = v = p / Pmax, so each MW
  costs e_g = c_g + (c_NL,g + c_SU,g) / Pmax_g; units fill in increasing e up
  to the demand and the rest is shed at VOLL.  The marginal price (LMP) is the
  e of the partly loaded unit.
* ``two_bus``: cheap unit at bus 0, expensive unit plus all load at bus 1, one
  line of limit F below the load: the line carries F, each bus is priced by
  its own unit, and the price difference is the line limit's shadow price.
* ``ptdf``: the DC flow identity f = diag(1/x) M_r B_r^{-1} inj_r, with M the
  line-bus incidence (+1 at from, -1 at to), B = M^T diag(1/x) M and the
  reference bus removed; inj = C p + s - d per period.
"""
from __future__ import annotations

import numpy as np


def merit_order(pmax, c_lin, c_nl, c_su, demand, voll):
    e = np.asarray(c_lin) + (np.asarray(c_nl) + np.asarray(c_su)) / np.asarray(pmax)
    order = np.argsort(e, kind="stable")
    p = np.zeros(len(e))
    left = float(demand)
    lmp = None
    for g in order:
        take = min(left, float(pmax[g]))
        p[g] = take
        left -= take
        if take < pmax[g] and take > 0:
            lmp = float(e[g])
        if left <= 0:
            if lmp is None:
                lmp = float(e[g])
            break
    shed = max(left, 0.0)
    if shed > 0:
        lmp = float(voll)
    obj = float(np.dot(e, p) + voll * shed)
    return obj, p, shed, lmp


def two_bus(e_cheap, pmax_cheap, e_exp, pmax_exp, demand, F):
    """Cheap unit at bus 0, expensive unit and load at bus 1; F < demand."""
    flow = min(F, pmax_cheap, demand)
    p_exp = demand - flow
    assert p_exp <= pmax_exp
    obj = e_cheap * flow + e_exp * p_exp
    return obj, flow, e_cheap, e_exp


def ptdf(P) -> np.ndarray:
    L, B = P.L, P.B
    M = np.zeros((L, B))
    M[np.arange(L), P.line_from] = 1.0
    M[np.arange(L), P.line_to] = -1.0
    Xi = np.diag(1.0 / P.x_pu)
    Bbus = M.T @ Xi @ M
    keep = np.array([b for b in range(B) if b != P.ref_bus])
    Br = Bbus[np.ix_(keep, keep)]
    out = np.zeros((L, B))
    out[:, keep] = Xi @ M[:, keep] @ np.linalg.inv(Br)
    return out


def injections(P, p, shed) -> np.ndarray:
    """[T, B] net injection C p + s - d."""
    inj = -P.load.copy()
    for g in range(P.G):
        inj[:, P.gen_bus[g]] += p[:, g]
    return inj + shed
