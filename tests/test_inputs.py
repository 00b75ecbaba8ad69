"""The seeded synthetic inputs follow the stated recipe: connected simple grids
(random spanning tree plus extra edges), parameter ranges, the load profile,
the served-request perturbation and Poisson arrivals.  CPU only."""
import math

import numpy as np
import pytest

import ucgen


def _connected(B, lf, lt):
    parent = list(range(B))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a
    for a, b in zip(lf, lt):
        parent[find(int(a))] = find(int(b))
    return len({find(i) for i in range(B)}) == 1


@pytest.mark.parametrize("make", [lambda: ucgen.tiny(0), lambda: ucgen.tiny(3),
                                  lambda: ucgen.make_problem(2, B=400, L=530, G=48, T=24, lo=0.5, hi=0.85,
                                                             noise=0.05, zero_pmin_frac=0.1)])
def test_grid_and_units_follow_the_recipe(make):
    P = make()
    assert len(P.line_from) == P.L and _connected(P.B, P.line_from, P.line_to)
    assert (P.line_from != P.line_to).all()
    pairs = {(min(a, b), max(a, b)) for a, b in zip(P.line_from.tolist(), P.line_to.tolist())}
    assert len(pairs) == P.L                                    # a simple graph
    assert ((0.01 <= P.x_pu) & (P.x_pu <= 0.2)).all() and ((50 <= P.fmax) & (P.fmax <= 200)).all()
    assert ((50 <= P.pmax) & (P.pmax <= 300)).all()
    on = P.pmin > 0
    np.testing.assert_allclose(P.pmin[on], 0.3 * P.pmax[on])
    np.testing.assert_allclose(P.ramp, 0.5 * P.pmax)
    assert ((10 <= P.c_lin) & (P.c_lin <= 60)).all() and ((100 <= P.c_nl) & (P.c_nl <= 500)).all()
    assert ((500 <= P.c_su) & (P.c_su <= 3000)).all() and (P.u0 == 0).all()
    assert ((0 <= P.gen_bus) & (P.gen_bus < P.B)).all()


def test_paper_scale_sizes_and_zero_pmin_share():
    P = ucgen.paper_scale(0)
    assert (P.B, P.L, P.G, P.T) == (6049, 8000, 700, 48) and _connected(P.B, P.line_from, P.line_to)
    assert int((P.pmin == 0).sum()) == 70                      # 10 % of the units


def test_load_profile_without_noise_is_the_stated_sinusoid():
    P = ucgen.tiny(1)
    cap = P.pmax.sum()
    t = np.arange(P.T)
    want = cap * (0.4 + 0.4 * 0.5 * (1 - np.cos(2 * math.pi * t / P.T)))
    np.testing.assert_allclose(P.load.sum(axis=1), want, rtol=1e-12)
    assert P.load.sum(axis=1).argmin() == 0                    # trough at t = 0
    share = P.load / P.load.sum(axis=1, keepdims=True)
    np.testing.assert_allclose(share, np.broadcast_to(share[0], share.shape), rtol=1e-10, atol=1e-15)   # one split


def test_generators_are_seeded():
    a, b = ucgen.paper_scale(0), ucgen.paper_scale(0)
    np.testing.assert_array_equal(a.load, b.load)
    np.testing.assert_array_equal(a.line_from, b.line_from)
    assert not np.array_equal(ucgen.tiny(0).load, ucgen.tiny(1).load)


def test_served_requests_scale_the_base_load():
    base = ucgen.tiny(0)
    scales = []
    for r in range(9):
        p = ucgen.served_request(base, 0, r)
        ratio = p.load.sum() / base.load.sum()
        scales.append(ucgen.LOAD_SCALES[r])
        assert abs(ratio - ucgen.LOAD_SCALES[r]) < 0.05 * ucgen.LOAD_SCALES[r]   # AR(1) noise of 5 %
        np.testing.assert_array_equal(p.pmax, base.pmax)       # same grid and units
    assert scales == [0.8, 0.85, 0.9, 0.95, 1.0, 1.05, 1.1, 1.15, 1.2]
    np.testing.assert_array_equal(ucgen.served_request(base, 2, 5).load, ucgen.served_request(base, 2, 5).load)


def test_poisson_arrivals_have_the_stated_rate():
    t = ucgen.poisson_arrivals(7, 20000, 2.0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all()
    assert abs(gaps.mean() - 0.5) < 0.02                       # 1 / rate
    assert abs(gaps.std() - 0.5) < 0.03                        # exponential: std = mean
