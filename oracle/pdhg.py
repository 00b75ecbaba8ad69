"""O1: restarted, diagonally scaled PDHG in plain FP64 numpy.

Test infrastructure only (see ``oracle/__init__``).

The paper's GPU arm solves the LP relaxation with PDHG (Sec. II-C, Alg. 1
"Solver 1"; Sec. III-C) with an iteration limit of 100,000, an absolute
feasibility tolerance of 1e-5 and a convergence tolerance of 1e-4 (Sec. II-D),
but does not state the method.  This follows the published PDLP scheme
(Applegate et al., NeurIPS 2021) with a constant step:

  start:  x = clip(0, l, u), y = 0, omega = omega0, tau = eta/omega,
          sigma = eta*omega, anchor = (x, y), KKT_anchor = KKT_omega(x, y)
  step k: x+ = clip(x - tau (c - A^T y), l, u)
          y+ = y + sigma (q - A (2 x+ - x)),  y+_I = max(y+_I, 0)
          running sums of x+, y+ since the last restart (uniform average)
  every n_eval steps (after step k with (k+1) % n_eval == 0):
          relative KKT (unscaled presolved LP) of the current point, then of
          the average: stop at the first one <= tol (current checked first);
          candidate = average if KKT_omega(avg) < KKT_omega(cur) else current;
          restart when KKT_c <= 0.2 KKT_anchor, or KKT_c <= 0.8 KKT_anchor and
          KKT_c > KKT_c at the previous evaluation, or j >= 0.36 (k+1)
          (j = steps since the last restart);
          on restart: dx = ||x_c - x_anchor||, dy = ||y_c - y_anchor||;
          if both > 1e-10, omega = exp(0.5 ln(dy/dx) + 0.5 ln omega);
          (x, y) = anchor = candidate; KKT_anchor = KKT_omega(candidate) with
          the new omega; sums and j reset; tau, sigma recomputed.
All arithmetic is on the scaled problem except the stopping test.

Adaptive step size (averaging variant, option ``adaptive=True``; PDLP,
Applegate et al. 2021, Sec. 3.1).  Each iteration is an attempt with the trial
step eta (initially the constant step S.eta):

  attempt: (x', y') = the PDHG step above with tau = eta/omega, sigma = eta*omega
           eta_bar = ||z' - z||^2_omega / (2 |(y' - y)^T A (x' - x)|)
                     (+inf when the product is 0), with
                     ||z||^2_omega = omega ||x||^2 + ||y||^2 / omega
           accepted when eta <= eta_bar: z = z', and z' enters the running
           sums with weight eta (the average is sum(eta z) / sum(eta));
           otherwise z stays
           next trial eta = min((1 - (k+1)^-0.3) eta_bar, (1 + (k+1)^-0.6) eta),
           k = attempts so far including this one (so k + 1 >= 2)
  Attempts count as iterations for the iteration limit, the evaluation period
  and the restart test's j; an evaluation with no accepted step since the
  last restart takes the current point as the average.

A second variant, the default, is restarted reflected Halpern PDHG (Lu &
Yang, "Restarted Halpern PDHG for linear programming", 2024), again with a
constant step.  With T the PDHG map above and z = (x, y):

  step:   z_hat = T(z)  (x_hat, y_hat as x+, y+ above, from the current z)
          z <- w (2 z_hat - z) + (1 - w) z0,   w = (j+1)/(j+2)
          (full reflection; z0 = anchor of the current restart epoch)
  every n_eval steps: relative KKT of z_hat (the last map output) -> stop;
          restart metric r = KKT_omega(z_hat) ("kkt"), the fixed-point
          residual sqrt(omega ||x_in - x_hat||^2 + ||y_in - y_hat||^2 / omega)
          of the last step ("fpr"), or that residual in the norm of the PDHG
          map's metric, sqrt(omega ||dx||^2 + ||dy||^2 / omega - 2 eta dy.A dx)
          with (dx, dy) = z_in - z_hat ("fprp": eta times the squared norm
          ||dx||^2 / tau + ||dy||^2 / sigma - 2 dy.A dx, in which the PDHG map
          is nonexpansive); the same three restart tests with r in
          place of KKT_c and r_anchor in place of KKT_anchor;
          on restart: omega from dx = ||x_hat - x0||, dy = ||y_hat - y0||,
          z = z0 = z_hat, j = 0, r_anchor = r re-weighted with the new omega.
The initial r_anchor is KKT_omega(z0) for "kkt" and +inf for "fpr" and "fprp".

The primal-weight update at a restart is PDLP's rule by default, written as a
proportional controller on ln omega (primal_weight_update, with the PID
generalisation as an option), optionally followed by a residual-balance guard
(guard_weight, option pw_guard): the new weight is kept only if it does not
move against the balance of the restart point's relative primal and dual
residuals by more than a factor kappa.

Primal feasibility polishing (after a solve that met the relative KKT
tolerance).  The paper's PDHG runs with an absolute feasibility tolerance of
1e-5 beside the 1e-4 convergence tolerance (Sec. II-D).  A point that meets
the relative test can still violate rows by more than that in absolute terms,
and on the UC LP such a violation (unserved load priced at VOLL) moves the
objective.  Polishing (PDLP's feasibility polishing, Applegate et al. 2025,
primal half) runs the Halpern variant on the feasibility problem -- the same
rows and bounds, objective c = 0 -- from the solve's primal point, a zero dual
and the solve's final primal weight, and stops when the map output's largest
absolute violation on the unscaled presolved LP (kkt.abs_primal_inf) is at
most the tolerance.  The polished primal replaces the solve's primal; the
solve's dual is kept.

Infeasibility detection (Halpern variant).  When the LP has no feasible point,
the map has no fixed point and the step residual T(z) - z tends to a nonzero
direction (the infimal displacement vector of the nonexpansive PDHG map).  At
every 4th evaluation, after the stopping test and before the restart test,
the dual part of the last step's residual, y_hat - y_in (mapped to the
unscaled LP), is tested as a Farkas direction (kkt.farkas_ray); when it passes,
the solve stops with status "infeasible".  The UC LP's feasible set is
bounded (every column has finite bounds or is tied to bounded columns), so
its objective cannot be unbounded and only this test is needed.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import kkt

BETA_SUFFICIENT = 0.2
BETA_NECESSARY = 0.8
BETA_ARTIFICIAL = 0.36
N_EVAL = 64


PDLP_GAINS = (0.5, 0.0, 0.0)
DEFAULT_PW_GAINS = PDLP_GAINS     # the gains the solves use unless told otherwise


@dataclasses.dataclass
class PrimalWeightControl:
    """PID controller on ln omega at restarts (see primal_weight_update)."""
    kp: float = 0.5
    ki: float = 0.0
    kd: float = 0.0
    isum: float = 0.0        # sum of the errors so far
    eprev: float = 0.0       # the last error
    has: bool = False        # an error was seen


@dataclasses.dataclass
class State:
    x: np.ndarray
    y: np.ndarray
    x_sum: np.ndarray
    y_sum: np.ndarray
    x_anchor: np.ndarray
    y_anchor: np.ndarray
    omega: float
    tau: float
    sigma: float
    kkt_anchor: float
    kkt_prev: float
    j: int
    k: int
    restarts: int = 0
    # adaptive step size
    eta_try: float = 0.0
    w_sum: float = 0.0
    accepted: int = 0
    pw: PrimalWeightControl = dataclasses.field(default_factory=PrimalWeightControl)


@dataclasses.dataclass
class Result:
    x: np.ndarray          # scaled presolved primal (returned point)
    y: np.ndarray          # scaled presolved dual
    iters: int
    status: str            # "optimal" | "iteration_limit" | "infeasible" (Halpern)
    rel: tuple             # (rel_p, rel_d, rel_gap) of the returned point
    restarts: int
    omega: float
    state: State
    which: str             # "current" | "average"


def _unscaled_lp(S):
    """The unscaled presolved LP, rebuilt from the scaled one and D_r, D_c."""
    class _U:
        pass
    U = _U()
    U.A = S.A.multiply(1.0 / S.Dr[:, None]).multiply(1.0 / S.Dc[None, :]).tocsr()
    U.q = S.q / S.Dr
    U.c = S.c / S.Dc
    with np.errstate(invalid="ignore"):
        U.l = S.l * S.Dc
        U.u = S.u * S.Dc
    U.m_eq = S.m_eq
    return U


def weighted(S, x, y, omega):
    r = kkt.residuals(S.A, S.q, S.c, S.l, S.u, S.m_eq, x, y)
    rp2 = float(np.dot(r.rp, r.rp))
    rd2 = float(np.dot(r.rd, r.rd))
    return kkt.weighted_kkt(rp2, rd2, r.gap, omega), (rp2, rd2, r.gap)


def initial_state(S, x0=None, y0=None) -> State:
    x = np.clip(np.zeros(S.A.shape[1]), S.l, S.u) if x0 is None else np.clip(x0.copy(), S.l, S.u)
    y = np.zeros(S.A.shape[0]) if y0 is None else y0.copy()
    if y0 is not None:
        y[S.m_eq:] = np.maximum(y[S.m_eq:], 0.0)
    omega = S.omega0
    ka, _ = weighted(S, x, y, omega)
    return State(x=x, y=y, x_sum=np.zeros_like(x), y_sum=np.zeros_like(y),
                 x_anchor=x.copy(), y_anchor=y.copy(), omega=omega,
                 tau=S.eta / omega, sigma=S.eta * omega, kkt_anchor=ka,
                 kkt_prev=math.inf, j=0, k=0, eta_try=S.eta)


def step(S, st: State, AT=None):
    """One PDHG iteration in place."""
    AT = S.A.T.tocsr() if AT is None else AT
    x_new = np.clip(st.x - st.tau * (S.c - AT @ st.y), S.l, S.u)
    xbar = 2.0 * x_new - st.x
    y_new = st.y + st.sigma * (S.q - S.A @ xbar)
    y_new[S.m_eq:] = np.maximum(y_new[S.m_eq:], 0.0)
    st.x = x_new
    st.y = y_new
    st.x_sum += x_new
    st.y_sum += y_new
    st.j += 1
    st.k += 1


ADAPT_SHRINK = 0.3    # exponent of the shrink factor 1 - (k+1)^-0.3
ADAPT_GROW = 0.6      # exponent of the growth factor 1 + (k+1)^-0.6


def adaptive_attempt(S, st: State, AT=None, exact_sums: bool = False):
    """One attempt of the adaptive step (PDLP, Applegate et al. 2021, Sec. 3.1),
    in place.  Returns (accepted, eta, eta_bar).  ``exact_sums`` takes the three
    sums of eta_bar correctly rounded (math.fsum) instead of numpy's order: the
    step feeds back into the next one, so comparing the two measures how far
    rounding alone moves the trajectory."""
    AT = S.A.T.tocsr() if AT is None else AT
    dot = (lambda a, b: math.fsum(a * b)) if exact_sums else (lambda a, b: float(np.dot(a, b)))
    eta = st.eta_try
    tau, sigma = eta / st.omega, eta * st.omega
    x_new = np.clip(st.x - tau * (S.c - AT @ st.y), S.l, S.u)
    y_new = st.y + sigma * (S.q - S.A @ (2.0 * x_new - st.x))
    y_new[S.m_eq:] = np.maximum(y_new[S.m_eq:], 0.0)
    dx = x_new - st.x
    dy = y_new - st.y
    movement = st.omega * dot(dx, dx) + dot(dy, dy) / st.omega
    interaction = abs(dot(dy, S.A @ dx))
    eta_bar = movement / (2.0 * interaction) if interaction > 0.0 else math.inf
    k = st.k + 1
    eta_next = min((1.0 - (k + 1) ** -ADAPT_SHRINK) * eta_bar, (1.0 + (k + 1) ** -ADAPT_GROW) * eta)
    accepted = eta <= eta_bar
    if accepted:
        st.x = x_new
        st.y = y_new
        st.x_sum += eta * x_new
        st.y_sum += eta * y_new
        st.w_sum += eta
        st.accepted += 1
    st.eta_try = eta_next
    st.j += 1
    st.k += 1
    return accepted, eta, eta_bar


def restart_decision(kkt_cand, kkt_anchor, kkt_prev, j, k_plus_1) -> bool:
    """The restart test applied at an evaluation (k_plus_1 = steps taken)."""
    if kkt_cand <= BETA_SUFFICIENT * kkt_anchor:
        return True
    if kkt_cand <= BETA_NECESSARY * kkt_anchor and kkt_cand > kkt_prev:
        return True
    if j >= BETA_ARTIFICIAL * k_plus_1:
        return True
    return False


def primal_weight_update(omega, dx, dy, ctl: PrimalWeightControl | None = None) -> float:
    """The primal weight after a restart whose epoch moved the primal by dx and
    the dual by dy.  The error e = ln(omega dx / dy) vanishes when the weighted
    movements omega dx^2 and dy^2 / omega balance; the update is
    ln omega <- ln omega - (kp e + ki sum(e) + kd (e - e_prev)) (the derivative
    term is 0 at the first update).  PDLP's rule (Applegate et al. 2021),
    omega <- exp(0.5 ln(dy/dx) + 0.5 ln omega), is kp = 0.5, ki = kd = 0, and is
    computed in that form.  omega is kept when dx or dy is at most 1e-10."""
    if not (dx > 1e-10 and dy > 1e-10):
        return omega
    if ctl is None or (ctl.kp, ctl.ki, ctl.kd) == PDLP_GAINS:
        return math.exp(0.5 * math.log(dy / dx) + 0.5 * math.log(omega))
    e = math.log(omega * dx / dy)
    ctl.isum += e
    de = e - ctl.eprev if ctl.has else 0.0
    ctl.eprev = e
    ctl.has = True
    return math.exp(math.log(omega) - (ctl.kp * e + ctl.ki * ctl.isum + ctl.kd * de))


def guard_weight(omega, omega_new, rel_p, rel_d, kappa) -> float:
    """Residual-balance guard on a primal-weight update.  A larger omega is a
    larger dual step sigma = eta omega, which works on primal infeasibility
    (the dual ascent direction is the primal residual), and a smaller omega a
    larger primal step, which works on dual infeasibility -- the residual
    balancing of ADMM and adaptive PDHG (Boyd et al. 2011, Sec. 3.4.1;
    Goldstein et al. 2015).  The controller's omega_new is dropped (omega kept)
    when it moves against the balance of the relative residuals of the restart
    point by more than the factor kappa: a decrease while rel_p > kappa rel_d,
    an increase while rel_d > kappa rel_p.  kappa = 0 turns the guard off."""
    if kappa > 0.0 and ((omega_new < omega and rel_p > kappa * rel_d) or
                        (omega_new > omega and rel_d > kappa * rel_p)):
        return omega
    return omega_new


def evaluate(S, st: State, U, tol: float, adaptive: bool = False):
    """Evaluation after an n_eval block; returns (done, which, point) and
    applies a restart to ``st`` when the test fires."""
    if not adaptive:
        x_avg = st.x_sum / st.j
        y_avg = st.y_sum / st.j
    elif st.w_sum > 0.0:
        x_avg = st.x_sum / st.w_sum
        y_avg = st.y_sum / st.w_sum
    else:   # no step accepted since the last restart
        x_avg = st.x
        y_avg = st.y
    for which, (xx, yy) in (("current", (st.x, st.y)), ("average", (x_avg, y_avg))):
        rel = kkt.relative_kkt(U, S.Dc * xx, S.Dr * yy)
        if max(rel) <= tol:
            return True, which, (xx.copy(), yy.copy()), rel
    k_cur, parts_cur = weighted(S, st.x, st.y, st.omega)
    k_avg, parts_avg = weighted(S, x_avg, y_avg, st.omega)
    if k_avg < k_cur:
        xc, yc, kc, parts = x_avg, y_avg, k_avg, parts_avg
    else:
        xc, yc, kc, parts = st.x, st.y, k_cur, parts_cur
    if restart_decision(kc, st.kkt_anchor, st.kkt_prev, st.j, st.k):
        dx = float(np.linalg.norm(xc - st.x_anchor))
        dy = float(np.linalg.norm(yc - st.y_anchor))
        st.omega = primal_weight_update(st.omega, dx, dy, st.pw)
        st.x = xc.copy()
        st.y = yc.copy()
        st.x_anchor = st.x.copy()
        st.y_anchor = st.y.copy()
        st.kkt_anchor = kkt.weighted_kkt(parts[0], parts[1], parts[2], st.omega)
        st.kkt_prev = math.inf
        st.x_sum[:] = 0.0
        st.y_sum[:] = 0.0
        st.w_sum = 0.0
        st.j = 0
        st.tau = S.eta / st.omega
        st.sigma = S.eta * st.omega
        st.restarts += 1
    else:
        st.kkt_prev = kc
    return False, None, None, None


def solve(S, tol: float = 1e-4, max_iter: int = 100_000, n_eval: int = N_EVAL,
          x0=None, y0=None, trace=None, trace_iters=(), adaptive: bool = False, attempts=None,
          exact_sums: bool = False, pw_gains=None) -> Result:
    """Run O1 on a ``presolve.Scaled`` problem.  ``trace(k, state)`` is called
    after every step k in ``trace_iters`` (k counts steps taken; with
    ``adaptive``, attempts).  ``attempts``, a list, receives (accepted, eta,
    eta_bar) of every adaptive attempt."""
    st = initial_state(S, x0, y0)
    st.pw = PrimalWeightControl(*(DEFAULT_PW_GAINS if pw_gains is None else pw_gains))
    AT = S.A.T.tocsr()
    U = _unscaled_lp(S)
    trace_iters = set(trace_iters)
    while st.k < max_iter:
        if adaptive:
            a = adaptive_attempt(S, st, AT, exact_sums)
            if attempts is not None:
                attempts.append(a)
        else:
            step(S, st, AT)
        if st.k % n_eval == 0:
            done, which, pt, rel = evaluate(S, st, U, tol, adaptive)
            if done:
                return Result(x=pt[0], y=pt[1], iters=st.k, status="optimal", rel=rel,
                              restarts=st.restarts, omega=st.omega, state=st, which=which)
        if trace is not None and st.k in trace_iters:
            trace(st.k, st)
    rel = kkt.relative_kkt(U, S.Dc * st.x, S.Dr * st.y)
    return Result(x=st.x.copy(), y=st.y.copy(), iters=st.k, status="iteration_limit",
                  rel=rel, restarts=st.restarts, omega=st.omega, state=st, which="current")


# ---------------------------------------------------------------------------
# restarted reflected Halpern PDHG (default variant)
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class HState:
    x: np.ndarray            # current Halpern iterate
    y: np.ndarray
    x0: np.ndarray           # epoch anchor
    y0: np.ndarray
    xh: np.ndarray           # last map output T(z)
    yh: np.ndarray
    x_in: np.ndarray         # input of the last step
    y_in: np.ndarray
    omega: float
    tau: float
    sigma: float
    r_anchor: float
    r_prev: float
    j: int
    k: int
    metric: str
    restarts: int = 0
    evals: int = 0
    pw: PrimalWeightControl = dataclasses.field(default_factory=PrimalWeightControl)
    pw_guard: float = 0.0    # residual-balance guard kappa (see guard_weight; 0: off)


INFEAS_EVERY = 4      # evaluations between infeasibility tests


def halpern_initial_state(S, x0=None, y0=None, metric: str = "kkt", omega0=None) -> HState:
    """Start point clip(x0, l, u), y0 with y_I >= 0 (zeros by default); the
    primal weight starts at omega0 when given (a warm start's weight), else
    at S.omega0."""
    x = np.clip(np.zeros(S.A.shape[1]) if x0 is None else x0.copy(), S.l, S.u)
    y = np.zeros(S.A.shape[0]) if y0 is None else y0.copy()
    y[S.m_eq:] = np.maximum(y[S.m_eq:], 0.0)
    omega = S.omega0 if omega0 is None else float(omega0)
    if metric == "kkt":
        ra, _ = weighted(S, x, y, omega)
    else:
        ra = math.inf
    return HState(x=x, y=y, x0=x.copy(), y0=y.copy(), xh=x.copy(), yh=y.copy(), x_in=x.copy(),
                  y_in=y.copy(), omega=omega, tau=S.eta / omega, sigma=S.eta * omega, r_anchor=ra,
                  r_prev=math.inf, j=0, k=0, metric=metric)


def halpern_step(S, st: HState, AT=None):
    AT = S.A.T.tocsr() if AT is None else AT
    xh = np.clip(st.x - st.tau * (S.c - AT @ st.y), S.l, S.u)
    xbar = 2.0 * xh - st.x
    yh = st.y + st.sigma * (S.q - S.A @ xbar)
    yh[S.m_eq:] = np.maximum(yh[S.m_eq:], 0.0)
    w = (st.j + 1) / (st.j + 2)
    x_new = w * xbar + (1.0 - w) * st.x0
    y_new = w * (2.0 * yh - st.y) + (1.0 - w) * st.y0
    st.x_in, st.y_in = st.x, st.y
    st.xh, st.yh = xh, yh
    st.x, st.y = x_new, y_new
    st.j += 1
    st.k += 1


def halpern_evaluate(S, st: HState, U, tol: float, stop_abs=None):
    """Evaluation after an n_eval block: (status, point, rel) with status None
    (continue), "optimal" or "infeasible" (point = the Farkas direction, scaled
    dual space); applies a restart.  With ``stop_abs`` the stopping test is the
    largest absolute primal violation of the map output (unscaled) instead of
    the relative KKT."""
    st.evals += 1
    rel = kkt.relative_kkt(U, S.Dc * st.xh, S.Dr * st.yh)
    done = (max(rel) <= tol) if stop_abs is None else (kkt.abs_primal_inf(U, S.Dc * st.xh) <= stop_abs)
    if done:
        return "optimal", (st.xh.copy(), st.yh.copy()), rel
    if st.evals % INFEAS_EVERY == 0:
        ray = st.yh - st.y_in
        if kkt.is_infeasibility_certificate(U, S.Dr * ray):
            return "infeasible", (np.zeros_like(st.xh), ray), rel
    w = st.omega
    fx2 = float(np.dot(st.x_in - st.xh, st.x_in - st.xh))
    fy2 = float(np.dot(st.y_in - st.yh, st.y_in - st.yh))
    cross = 0.0
    if st.metric == "fprp":
        cross = float(np.dot(st.y_in - st.yh, S.A @ (st.x_in - st.xh)))
    if st.metric == "kkt":
        r, parts = weighted(S, st.xh, st.yh, w)
    else:
        r = math.sqrt(max(w * fx2 + fy2 / w - 2.0 * S.eta * cross, 0.0))
    if restart_decision(r, st.r_anchor, st.r_prev, st.j, st.k):
        dx = float(np.linalg.norm(st.xh - st.x0))
        dy = float(np.linalg.norm(st.yh - st.y0))
        st.omega = guard_weight(w, primal_weight_update(w, dx, dy, st.pw), rel[0], rel[1], st.pw_guard)
        wn = st.omega
        st.x = st.xh.copy()
        st.y = st.yh.copy()
        st.x0 = st.x.copy()
        st.y0 = st.y.copy()
        st.r_anchor = (kkt.weighted_kkt(parts[0], parts[1], parts[2], wn) if st.metric == "kkt"
                       else math.sqrt(max(wn * fx2 + fy2 / wn - 2.0 * S.eta * cross, 0.0)))
        st.r_prev = math.inf
        st.j = 0
        st.tau = S.eta / wn
        st.sigma = S.eta * wn
        st.restarts += 1
    else:
        st.r_prev = r
    return None, None, rel


def solve_halpern(S, tol: float = 1e-4, max_iter: int = 100_000, n_eval: int = N_EVAL,
                  x0=None, y0=None, metric: str = "kkt", trace=None, trace_iters=(),
                  omega0=None, stop_abs=None, pw_gains=None, pw_guard: float = 0.0) -> Result:
    """Run the Halpern variant; ``trace(k, state)`` after every step k in trace_iters
    (after the evaluation when k is a multiple of n_eval)."""
    st = halpern_initial_state(S, x0, y0, metric, omega0)
    st.pw = PrimalWeightControl(*(DEFAULT_PW_GAINS if pw_gains is None else pw_gains))
    st.pw_guard = float(pw_guard)
    AT = S.A.T.tocsr()
    U = _unscaled_lp(S)
    trace_iters = set(trace_iters)
    while st.k < max_iter:
        halpern_step(S, st, AT)
        if st.k % n_eval == 0:
            status, pt, rel = halpern_evaluate(S, st, U, tol, stop_abs)
            if status is not None:
                return Result(x=pt[0], y=pt[1], iters=st.k, status=status, rel=rel,
                              restarts=st.restarts, omega=st.omega, state=st,
                              which="map" if status == "optimal" else "ray")
        if trace is not None and st.k in trace_iters:
            trace(st.k, st)
    rel = kkt.relative_kkt(U, S.Dc * st.xh, S.Dr * st.yh)
    return Result(x=st.xh.copy(), y=st.yh.copy(), iters=st.k, status="iteration_limit", rel=rel,
                  restarts=st.restarts, omega=st.omega, state=st, which="map")


def polish_primal(S, x, tol_abs: float = 1e-5, max_iter: int = 10_000, omega0=None,
                  n_eval: int = N_EVAL, metric: str = "kkt", pw_gains=None, pw_guard: float = 0.0) -> Result:
    """Primal feasibility polishing (see the module docstring): the Halpern
    variant on the feasibility problem (c = 0) from the scaled primal ``x``, a
    zero dual and primal weight ``omega0`` (S.omega0 when None), until the
    largest absolute violation of the unscaled rows is <= ``tol_abs``."""
    F = dataclasses.replace(S, c=np.zeros_like(S.c))
    return solve_halpern(F, tol=0.0, max_iter=max_iter, n_eval=n_eval, x0=x, metric=metric,
                         omega0=omega0, stop_abs=tol_abs, pw_gains=pw_gains, pw_guard=pw_guard)
