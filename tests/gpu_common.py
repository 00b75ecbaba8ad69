"""Shared helpers of the GPU parity tests (not collected by pytest)."""
import json
import os

import numpy as np

from oracle import kkt, lp as olp, pdhg, presolve as ops

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# Per-iterate agreement of the FP64 device path with the FP64 oracle PDHG:
# both run the same arithmetic and differ only in summation order and FMA
# contraction (about 1e-16 relative per step); PDHG steps are non-expansive,
# so 1e-9 relative over the first few hundred iterations leaves a wide margin.
ITERATE_RTOL = 1e-9
KKT_TOL = 1e-4          # relative KKT (infinity norm), the paper's convergence tolerance
OBJ_GAP_TOL = 1e-4      # |obj - obj_simplex| / max(1, |obj_simplex|)


def golden_tiny():
    with open(os.path.join(GOLDEN, "tiny_lp.json")) as f:
        return json.load(f)


def oracle_pipeline(P):
    raw = olp.build_lp(P)
    ps = ops.presolve(raw)
    S = ops.scale(ps.lp)
    return raw, ps, S


def oracle_trace(S, ks, n_eval=pdhg.N_EVAL, variant="halpern", metric="kkt", **kw):
    """Oracle current iterates after each step count in ks (tol 0: never stops):
    {k: (x, y, restarts, omega, x_map, y_map)}; x_map/y_map are the last PDHG
    map output for the Halpern variant (None for the averaging variant)."""
    out = {}
    def rec(k, st):
        xm = getattr(st, "xh", None)
        ym = getattr(st, "yh", None)
        out[k] = (st.x.copy(), st.y.copy(), st.restarts, st.omega,
                  None if xm is None else xm.copy(), None if ym is None else ym.copy())
    if variant == "halpern":
        pdhg.solve_halpern(S, tol=0.0, max_iter=max(ks), n_eval=n_eval, metric=metric, trace=rec,
                           trace_iters=ks, **kw)
    else:
        pdhg.solve(S, tol=0.0, max_iter=max(ks), n_eval=n_eval, trace=rec, trace_iters=ks)
    return out


def oracle_solve(S, tol, variant="halpern", metric="kkt", **kw):
    if variant == "halpern":
        return pdhg.solve_halpern(S, tol=tol, metric=metric, **kw)
    return pdhg.solve(S, tol=tol)


def rel_inf(a, b):
    d = np.max(np.abs(a - b), initial=0.0)
    r = np.max(np.abs(b), initial=0.0)
    return d / r if r > 0 else d


def oracle_kkt_of_raw(ps, xr, yr):
    """Relative KKT, as the oracle computes it, of a raw-LP point mapped to the
    oracle's presolved LP."""
    return kkt.relative_kkt(ps.lp, xr[ps.col_map], yr[ps.row_map])


def raw_objective(raw, xr):
    return float(raw.c @ xr)
