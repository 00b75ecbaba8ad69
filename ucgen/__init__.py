"""Seeded synthetic unit-commitment instances.

This module only draws problem DATA (network, units, loads) from seeded random
streams.  It contains none of the solver's arithmetic: no LP rows, no presolve,
no scaling, no PDHG.  Both the CUDA product path and the CPU oracle take their
inputs from here, and nothing else is shared between them.

The paper evaluates on the ARPA-E GO Challenge 3 6,049-bus cases (Sec. II-E,
Table I), which are not available; these generators stand in for them with the
same bus count, the D2 horizon of 48 periods (Sec. II-D) and the
millions-of-variables scale.  The recipe:

* network: a random spanning tree (decoded from a uniform Pruefer sequence)
  plus uniformly drawn extra edges between non-adjacent bus pairs until there
  are ``L`` lines; reactance x ~ U[0.01, 0.2] p.u., limit F ~ U[50, 200] MW;
* units: bus uniform with replacement, Pmax ~ U[50, 300] MW, Pmin = 0.3 Pmax
  (a fraction of units gets Pmin = 0), ramp = 0.5 Pmax per period, linear cost
  ~ U[10, 60] $/MWh, no-load ~ U[100, 500] $, startup ~ U[500, 3000] $, all
  initially off;
* load: the system total follows a daily sinusoid between ``lo`` and ``hi``
  times total capacity (trough at t = 0), split over buses by one Dirichlet(1)
  draw, optionally with per-(bus, period) multiplicative Gaussian noise or an
  AR(1) perturbation, clipped at zero.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "UCProblem", "make_grid", "make_units", "make_load", "make_problem",
    "tiny", "micro", "paper_scale", "batch_member", "served_request",
]

DEFAULT_VOLL = 10_000.0


@dataclasses.dataclass
class UCProblem:
    """Raw DC unit-commitment data (all arrays numpy, contiguous)."""
    B: int
    L: int
    G: int
    T: int
    ref_bus: int
    line_from: np.ndarray  # int32 [L]
    line_to: np.ndarray    # int32 [L]
    x_pu: np.ndarray       # f64 [L] reactance, p.u.
    fmax: np.ndarray       # f64 [L] MW
    gen_bus: np.ndarray    # int32 [G]
    pmax: np.ndarray       # f64 [G] MW
    pmin: np.ndarray       # f64 [G] MW
    ramp: np.ndarray       # f64 [G] MW / period
    c_lin: np.ndarray      # f64 [G] $/MWh
    c_nl: np.ndarray       # f64 [G] $ per committed period
    c_su: np.ndarray       # f64 [G] $ per startup
    u0: np.ndarray         # f64 [G] initial commitment (0 or 1)
    load: np.ndarray       # f64 [T, B] MW, time-major
    voll: float = DEFAULT_VOLL
    name: str = ""

    def copy(self) -> "UCProblem":
        return dataclasses.replace(
            self, **{f.name: (getattr(self, f.name).copy()
                              if isinstance(getattr(self, f.name), np.ndarray)
                              else getattr(self, f.name))
                     for f in dataclasses.fields(self)})


def _pruefer_tree(rng: np.random.Generator, B: int) -> list[tuple[int, int]]:
    """Uniform random labelled tree on B nodes via a random Pruefer sequence."""
    if B == 1:
        return []
    if B == 2:
        return [(0, 1)]
    seq = rng.integers(0, B, size=B - 2)
    degree = np.ones(B, dtype=np.int64)
    for s in seq:
        degree[s] += 1
    import heapq
    leaves = [i for i in range(B) if degree[i] == 1]
    heapq.heapify(leaves)
    edges = []
    for s in seq:
        leaf = heapq.heappop(leaves)
        edges.append((leaf, int(s)))
        degree[s] -= 1
        if degree[s] == 1:
            heapq.heappush(leaves, int(s))
    a = heapq.heappop(leaves)
    b = heapq.heappop(leaves)
    edges.append((a, b))
    return edges


def make_grid(rng: np.random.Generator, B: int, L: int):
    """Connected random network: spanning tree plus extra distinct edges."""
    if L < B - 1:
        raise ValueError("need at least B-1 lines for a connected grid")
    max_edges = B * (B - 1) // 2
    if L > max_edges:
        raise ValueError("too many lines for a simple graph")
    edges = _pruefer_tree(rng, B)
    seen = {(min(a, b), max(a, b)) for a, b in edges}
    while len(edges) < L:
        need = L - len(edges)
        cand = rng.integers(0, B, size=(2 * need + 8, 2))
        for a, b in cand:
            if a == b:
                continue
            key = (int(min(a, b)), int(max(a, b)))
            if key in seen:
                continue
            seen.add(key)
            edges.append((int(a), int(b)))
            if len(edges) == L:
                break
    e = np.asarray(edges, dtype=np.int32).reshape(-1, 2)
    x = rng.uniform(0.01, 0.2, size=L)
    fmax = rng.uniform(50.0, 200.0, size=L)
    return e[:, 0].copy(), e[:, 1].copy(), x, fmax


def make_units(rng: np.random.Generator, G: int, B: int, zero_pmin_frac: float = 0.0):
    gen_bus = rng.integers(0, B, size=G).astype(np.int32)
    pmax = rng.uniform(50.0, 300.0, size=G)
    pmin = 0.3 * pmax
    if zero_pmin_frac > 0.0:
        k = int(round(zero_pmin_frac * G))
        idx = rng.choice(G, size=k, replace=False)
        pmin[idx] = 0.0
    ramp = 0.5 * pmax
    c_lin = rng.uniform(10.0, 60.0, size=G)
    c_nl = rng.uniform(100.0, 500.0, size=G)
    c_su = rng.uniform(500.0, 3000.0, size=G)
    u0 = np.zeros(G)
    return gen_bus, pmax, pmin, ramp, c_lin, c_nl, c_su, u0


def make_load(rng: np.random.Generator, B: int, T: int, total_cap: float,
              lo: float, hi: float, noise: float = 0.0,
              ar1_rho: float | None = None, scale: float = 1.0) -> np.ndarray:
    """[T, B] MW.  noise: std of the multiplicative per-(b,t) perturbation;
    with ar1_rho set, the perturbation is a stationary AR(1) process over t."""
    t = np.arange(T, dtype=np.float64)
    shape = lo + (hi - lo) * 0.5 * (1.0 - np.cos(2.0 * math.pi * t / T))
    total = total_cap * shape * scale
    share = rng.dirichlet(np.ones(B))
    load = total[:, None] * share[None, :]
    if noise > 0.0:
        if ar1_rho is None:
            eps = rng.standard_normal((T, B))
            load = load * (1.0 + noise * eps)
        else:
            e = np.empty((T, B))
            e[0] = noise * rng.standard_normal(B)
            k = noise * math.sqrt(1.0 - ar1_rho * ar1_rho)
            for tt in range(1, T):
                e[tt] = ar1_rho * e[tt - 1] + k * rng.standard_normal(B)
            load = load * (1.0 + e)
    return np.ascontiguousarray(np.maximum(load, 0.0))


def make_problem(seed: int, B: int, L: int, G: int, T: int, lo: float, hi: float,
                 noise: float = 0.0, zero_pmin_frac: float = 0.0,
                 voll: float = DEFAULT_VOLL, name: str = "") -> UCProblem:
    rng = np.random.default_rng(seed)
    lf, lt, x, fmax = make_grid(rng, B, L)
    gen_bus, pmax, pmin, ramp, c_lin, c_nl, c_su, u0 = make_units(rng, G, B, zero_pmin_frac)
    load = make_load(rng, B, T, float(pmax.sum()), lo, hi, noise)
    return UCProblem(B=B, L=L, G=G, T=T, ref_bus=0, line_from=lf, line_to=lt,
                     x_pu=x, fmax=fmax, gen_bus=gen_bus, pmax=pmax, pmin=pmin,
                     ramp=ramp, c_lin=c_lin, c_nl=c_nl, c_su=c_su, u0=u0,
                     load=load, voll=voll, name=name)


def tiny(seed: int = 0, voll: float = DEFAULT_VOLL) -> UCProblem:
    """30 buses, 41 lines, 6 units, 24 hourly periods, load 0.4-0.8 of capacity."""
    return make_problem(seed, B=30, L=41, G=6, T=24, lo=0.4, hi=0.8, voll=voll,
                        name=f"tiny-30bus-s{seed}")


def micro(seed: int, B: int = 2, L: int = 1, G: int = 2, T: int = 2,
          lo: float = 0.4, hi: float = 0.8, voll: float = DEFAULT_VOLL) -> UCProblem:
    """Very small instance for brute force (commitments and vertices)."""
    return make_problem(seed, B=B, L=L, G=G, T=T, lo=lo, hi=hi, voll=voll,
                        name=f"micro-{B}b{G}g{T}t-s{seed}")


def paper_scale(seed: int = 0, B: int = 6049, L: int = 8000, G: int = 700, T: int = 48,
                voll: float = DEFAULT_VOLL) -> UCProblem:
    """6,049-bus / 8,000-line / 700-unit / 48-period instance, 10% zero-Pmin units,
    load 0.5-0.85 of capacity with 5% per-(bus, period) Gaussian noise."""
    return make_problem(seed, B=B, L=L, G=G, T=T, lo=0.5, hi=0.85, noise=0.05,
                        zero_pmin_frac=0.10, voll=voll, name=f"grid{B}-T{T}-s{seed}")


def batch_member(seed: int, voll: float = DEFAULT_VOLL) -> UCProblem:
    """One member of the uneven batch: B log-uniform in [300, 6049], L = 1.32 B,
    G = 0.12 B, T = 24 for odd seeds and 48 for even seeds."""
    rng = np.random.default_rng(10_000 + seed)
    B = int(round(math.exp(rng.uniform(math.log(300), math.log(6049)))))
    L = int(round(1.32 * B))
    G = max(1, int(round(0.12 * B)))
    T = 48 if seed % 2 == 0 else 24
    return make_problem(seed, B=B, L=L, G=G, T=T, lo=0.5, hi=0.85, noise=0.05,
                        zero_pmin_frac=0.10, voll=voll, name=f"batch-{B}b-T{T}-s{seed}")


LOAD_SCALES = tuple(round(0.80 + 0.05 * i, 2) for i in range(9))


def served_request(base: UCProblem, wave: int, r: int) -> UCProblem:
    """Request r of wave w: the base network and units with the load scaled by
    one of {0.80, ..., 1.20} and an AR(1) perturbation (sigma 5%, rho 0.9)."""
    seed = 1000 * wave + r
    rng = np.random.default_rng(seed)
    scale = LOAD_SCALES[r % len(LOAD_SCALES)]
    T, B = base.load.shape
    e = np.empty((T, B))
    sigma, rho = 0.05, 0.9
    e[0] = sigma * rng.standard_normal(B)
    k = sigma * math.sqrt(1.0 - rho * rho)
    for tt in range(1, T):
        e[tt] = rho * e[tt - 1] + k * rng.standard_normal(B)
    p = base.copy()
    p.load = np.ascontiguousarray(np.maximum(base.load * scale * (1.0 + e), 0.0))
    p.name = f"{base.name}-w{wave}r{r}x{scale:.2f}"
    return p


def poisson_arrivals(seed: int, n: int, rate: float) -> np.ndarray:
    """Arrival times (s) of n requests of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))
