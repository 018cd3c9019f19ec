"""Pins for the oracle's error bounds, order selection, distance bounds and
method choice (Sections 2.2, 3.4, 3.5)."""
import math

import mpmath as mp
import numpy as np
import pytest

mp.mp.dps = 50


@pytest.mark.parametrize("D", [1, 2, 3, 5, 8])
def test_farfield_bound_binomial_closed_form(orc, D):
    # sum_{k<D} C(D,k) a^k b^{D-k} = (a+b)^D - a^D with a = 1-r^p, b = r^p/sqrt(p!).
    for r in (0.05, 0.3, 0.7, 0.95):
        for p in range(1, 7):
            R = mp.mpf(r)
            a = 1 - R ** p
            b = R ** p / mp.sqrt(mp.factorial(p))
            want = float(17 / (1 - R) ** D * ((a + b) ** D - a ** D))
            got = orc.bound_farfield(17.0, D, r, p)
            assert got == pytest.approx(want, rel=1e-9, abs=1e-300)
            assert orc.bound_local(17.0, D, r, p) == got


@pytest.mark.parametrize("D", [1, 2, 3, 5])
def test_f2l_bound_binomial_closed_form(orc, D):
    for r in (0.05, 0.2, 0.45):
        for p in range(1, 7):
            q = (2 * mp.mpf(r)) ** p
            a = (1 - q) ** 2
            b = q * (2 - q) / mp.sqrt(mp.factorial(p))
            want = float(5 / (1 - 2 * mp.mpf(r)) ** (2 * D) * ((a + b) ** D - a ** D))
            assert orc.bound_f2l(5.0, D, r, p) == pytest.approx(want, rel=1e-9, abs=1e-300)


def test_bounds_scale_with_node_size_and_vanish(orc):
    for D in (1, 2, 3, 5):
        for r in (0.1, 0.4):
            vals = [orc.bound_farfield(1.0, D, r, p) for p in range(1, 12)]
            assert all(b > a for a, b in zip(vals[1:], vals[:-1]))  # decreasing in p
            assert vals[-1] < 1e-6
            assert orc.bound_farfield(2.0, D, r, 3) == pytest.approx(2 * orc.bound_farfield(1.0, D, r, 3))


def test_orders_infinite_for_large_nodes_and_least_order(orc):
    D, h, pm = 3, 0.1, 4
    lo = np.zeros(D)
    # side 2h -> r = 1: far field / local impossible
    assert orc.order_farfield(lo, lo + 2 * h, 10, h, 1e9, pm) == orc.INF_ORDER
    assert orc.order_local(lo, lo + 2 * h, 10, h, 1e9, pm) == orc.INF_ORDER
    # side h -> r = 1/2: far-to-local impossible, far field possible
    assert orc.order_f2l(lo, lo + h, lo, lo + 0.1 * h, 10, h, 1e9, pm) == orc.INF_ORDER
    assert orc.order_farfield(lo, lo + h, 10, h, 1e9, pm) == 1
    # least order meeting tau
    r = 0.3
    side = 2 * r * h
    for tau_p in range(1, pm + 1):
        tau = orc.bound_farfield(10, D, r, tau_p)
        p = orc.order_farfield(lo, lo + side, 10, h, tau * (1 + 1e-12), pm)
        assert p == tau_p
    # bound above tau at p_max -> infinite
    assert orc.order_farfield(lo, lo + side, 10, h, 1e-30, pm) == orc.INF_ORDER


def test_distance_bounds_brute_force(orc):
    rng = np.random.default_rng(7)
    for D in (1, 2, 3, 6):
        for _ in range(30):
            a = rng.random((2, D))
            b = rng.random((2, D)) + rng.uniform(-1, 1)
            Ql, Qu = a.min(0), a.max(0)
            Rl, Ru = b.min(0), b.max(0)
            dl, du = orc.dist_bounds(Ql, Qu, Rl, Ru)
            q = rng.uniform(Ql, Qu, size=(200, D))
            r = rng.uniform(Rl, Ru, size=(200, D))
            dist = np.linalg.norm(q[:, None] - r[None], axis=2)
            assert dist.min() >= dl - 1e-12 and dist.max() <= du + 1e-12
            # attained at box corners
            corners_q = np.array(np.meshgrid(*[[Ql[d], Qu[d]] for d in range(D)])).reshape(D, -1).T
            corners_r = np.array(np.meshgrid(*[[Rl[d], Ru[d]] for d in range(D)])).reshape(D, -1).T
            cd = np.linalg.norm(corners_q[:, None] - corners_r[None], axis=2)
            assert cd.max() == pytest.approx(du, rel=1e-12)
            overlap = np.all((Ql <= Ru) & (Rl <= Qu))
            if overlap:
                assert dl == 0.0
            else:
                gap = np.maximum(0, np.maximum(Rl - Qu, Ql - Ru))
                assert dl == pytest.approx(np.linalg.norm(gap), rel=1e-12)


def test_choose_best_method(orc):
    D, h, pm = 3, 1.0, 4
    lo = np.zeros(D)
    small = lo + 0.05
    # large reference node, few queries: far-field evaluation wins
    m, p = orc.choose_best_method(lo, small, 4, lo, small, 10_000, h, 1e3, pm)
    assert m == orc.METHOD_F and p >= 1
    # many queries, few references, order 3 needed: direct local accumulation wins
    m, p = orc.choose_best_method(lo, small, 10_000, lo, small, 4, h, 1e-3, pm)
    assert m == orc.METHOD_D
    # many of both: far-to-local translation wins
    m, p = orc.choose_best_method(lo, small, 10_000, lo, small, 10_000, h, 1e6, pm)
    assert m == orc.METHOD_T
    # boxes too large for any expansion: exhaustive (recurse)
    big = lo + 5.0
    m, p = orc.choose_best_method(lo, big, 100, lo, big, 100, h, 1e3, pm)
    assert m == orc.METHOD_E
    # tolerance too tight for any order up to p_max: exhaustive
    m, p = orc.choose_best_method(lo, small, 50, lo, small, 50, h, 1e-12, pm)
    assert m == orc.METHOD_E
    # tiny pair with a loose tolerance: the order-1 translation costs D,
    # less than the D N_Q N_R of the exhaustive sum
    m, p = orc.choose_best_method(lo, small, 2, lo, small, 2, h, 1e3, pm)
    assert m == orc.METHOD_T and p == 1
