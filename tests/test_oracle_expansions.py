"""Pins for the oracle's series expansions and translations (Sections 3.3-3.5).

Each truncated expansion is checked against the exact sum (itself pinned
in test_oracle_naive.py): its error stays under the paper's truncation
lemma and vanishes as the order grows.  The multi-index sums are also
checked against the per-dimension product form written with 1-D sums,
which catches a transposed or mis-ordered multi-index.  Far-to-far and
local-to-local translation are exact and checked as such.
"""
import math

import numpy as np
import pytest

from conftest import read_golden


def box_points(rng, n, c, w):
    return c + rng.uniform(-w, w, size=(n, len(c)))


# ------------------------------------------------------------ layout
@pytest.mark.parametrize("p,D", [(1, 1), (8, 1), (6, 2), (4, 3), (2, 5), (3, 4)])
def test_multi_index_bijection(orc, p, D):
    seen = set()
    for i in range(p ** D):
        a = orc.pos_to_multi(i, p, D)
        assert (a >= 0).all() and (a < p).all()
        assert orc.multi_to_pos(a, p) == i
        seen.add(tuple(a))
    assert len(seen) == p ** D


def test_multi_index_last_dimension_least_significant(orc):
    # MultiIndexToPosition walks d = D..1 with the place value growing by p.
    p, D = 4, 3
    assert orc.multi_to_pos([0, 0, 1], p) == 1
    assert orc.multi_to_pos([0, 1, 0], p) == p
    assert orc.multi_to_pos([1, 0, 0], p) == p * p


def test_pmax_table(orc):
    for D, pm in read_golden("pmax_table.txt"):
        assert orc.pmax(int(D)) == int(pm)


# ------------------------------------------------------------ far field
@pytest.mark.parametrize("D,r", [(1, 0.6), (2, 0.5), (2, 0.9), (3, 0.4), (3, 0.8), (5, 0.3)])
def test_farfield_within_lemma_and_converges(orc, D, r):
    rng = np.random.default_rng(10 + D)
    h = 0.07
    c = rng.random(D)
    R = box_points(rng, 60, c, 0.999 * r * h)
    q = np.concatenate([box_points(rng, 30, c, 4 * h), c + rng.normal(size=(10, D)) * 10 * h])
    exact = orc.naive_kde(q, R, h)
    for p in range(1, 7):
        M = orc.farfield_moments(R, c, h, p)
        approx = orc.eval_farfield(M, c, h, p, q)
        bound = orc.bound_farfield(len(R), D, r, p)
        assert np.all(np.abs(approx - exact) <= bound * (1 + 1e-9) + 1e-12)
    p = 24 if D <= 2 else (12 if D == 3 else 8)
    M = orc.farfield_moments(R, c, h, p)
    approx = orc.eval_farfield(M, c, h, p, q)
    err = np.max(np.abs(approx - exact))
    assert err <= orc.bound_farfield(len(R), D, r, p) * (1 + 1e-9) + 1e-12
    if orc.bound_farfield(1.0, D, r, p) < 1e-9:
        assert err < 1e-8 * len(R)


@pytest.mark.parametrize("D,p", [(2, 5), (3, 4)])
def test_farfield_matches_product_form(orc, D, p):
    # G~_F(q) = sum_r prod_d sum_{n<p} (1/n!) ((r_d-c_d)s)^n h_n((q_d-c_d)s)
    rng = np.random.default_rng(20 + D)
    h = 0.1
    s = 1 / math.sqrt(2 * h * h)
    c = rng.random(D)
    R = box_points(rng, 15, c, 0.08)
    q = box_points(rng, 12, c, 0.4)
    M = orc.farfield_moments(R, c, h, p)
    got = orc.eval_farfield(M, c, h, p, q)
    want = np.zeros(len(q))
    for i in range(len(q)):
        tot = 0.0
        for r in R:
            prod = 1.0
            for d in range(D):
                hn = orc.hermite_functions((q[i, d] - c[d]) * s, p)
                prod *= sum(((r[d] - c[d]) * s) ** n / math.factorial(n) * hn[n] for n in range(p))
            tot += prod
        want[i] = tot
    assert np.allclose(got, want, rtol=1e-12, atol=1e-13)


# ------------------------------------------------------------ local
@pytest.mark.parametrize("D,r", [(1, 0.7), (2, 0.5), (3, 0.45), (4, 0.3), (5, 0.25)])
def test_direct_local_within_lemma_and_converges(orc, D, r):
    rng = np.random.default_rng(30 + D)
    h = 0.05
    c = rng.random(D)
    Q = box_points(rng, 25, c, 0.999 * r * h)
    R = np.concatenate([box_points(rng, 40, c, 3 * h), c + rng.normal(size=(10, D)) * 6 * h])
    exact = orc.naive_kde(Q, R, h)
    for p in range(1, 7):
        L = orc.direct_local(R, c, h, p)
        approx = orc.eval_local(L, c, h, p, Q)
        bound = orc.bound_local(len(R), D, r, p)
        assert np.all(np.abs(approx - exact) <= bound * (1 + 1e-9) + 1e-12)
    p = 24 if D <= 2 else (12 if D == 3 else 8)
    L = orc.direct_local(R, c, h, p)
    approx = orc.eval_local(L, c, h, p, Q)
    err = np.max(np.abs(approx - exact))
    assert err <= orc.bound_local(len(R), D, r, p) * (1 + 1e-9) + 1e-12
    if orc.bound_local(1.0, D, r, p) < 1e-9:
        assert err < 1e-8 * len(R)


def test_direct_local_matches_product_form(orc):
    # sum_r prod_d sum_{n<p} ((-1)^n/n!) h_n((c_d-r_d)s) ((q_d-c_d)s)^n
    D, p, h = 3, 4, 0.1
    s = 1 / math.sqrt(2 * h * h)
    rng = np.random.default_rng(41)
    c = rng.random(D)
    R = box_points(rng, 10, c, 0.3)
    Q = box_points(rng, 8, c, 0.05)
    L = orc.direct_local(R, c, h, p)
    got = orc.eval_local(L, c, h, p, Q)
    want = np.zeros(len(Q))
    for i in range(len(Q)):
        for r in R:
            prod = 1.0
            for d in range(D):
                hn = orc.hermite_functions((c[d] - r[d]) * s, p)
                prod *= sum((-1) ** n / math.factorial(n) * hn[n] * ((Q[i, d] - c[d]) * s) ** n
                            for n in range(p))
            want[i] += prod
    assert np.allclose(got, want, rtol=1e-12, atol=1e-13)


# ------------------------------------------------------------ far to local
@pytest.mark.parametrize("D,r", [(1, 0.3), (2, 0.2), (2, 0.4), (3, 0.25), (5, 0.15)])
def test_far_to_local_within_lemma_and_converges(orc, D, r):
    rng = np.random.default_rng(50 + D)
    h = 0.08
    cR = rng.random(D)
    cQ = cR + rng.uniform(-3, 3, size=D) * h
    R = box_points(rng, 50, cR, 0.999 * r * h)
    Q = box_points(rng, 20, cQ, 0.999 * r * h)
    exact = orc.naive_kde(Q, R, h)
    for p in range(1, 6):
        M = orc.farfield_moments(R, cR, h, p)
        L = orc.far_to_local(M, cR, cQ, h, p)
        approx = orc.eval_local(L, cQ, h, p, Q)
        bound = orc.bound_f2l(len(R), D, r, p)
        assert np.all(np.abs(approx - exact) <= bound * (1 + 1e-9) + 1e-12)
    p = 16 if D <= 2 else (8 if D == 3 else 5)
    M = orc.farfield_moments(R, cR, h, p)
    L = orc.far_to_local(M, cR, cQ, h, p)
    approx = orc.eval_local(L, cQ, h, p, Q)
    err = np.max(np.abs(approx - exact))
    assert err <= orc.bound_f2l(len(R), D, r, p) * (1 + 1e-9) + 1e-12
    if orc.bound_f2l(1.0, D, r, p) < 1e-8:
        assert err < 1e-7 * len(R)


# ------------------------------------------------------------ translations
@pytest.mark.parametrize("D,p", [(1, 8), (2, 6), (3, 4), (5, 2)])
def test_far_to_far_is_exact(orc, D, p):
    # Moments of R = R1 u R2 about the parent center, built by translating
    # each child's moments, equal the moments computed from the points.
    rng = np.random.default_rng(60 + D)
    h = 0.05
    c1, c2 = rng.random(D), rng.random(D)
    R1 = box_points(rng, 30, c1, 0.03)
    R2 = box_points(rng, 20, c2, 0.02)
    R = np.concatenate([R1, R2])
    cp = 0.5 * (R.min(0) + R.max(0))
    M1 = orc.farfield_moments(R1, c1, h, p)
    M2 = orc.farfield_moments(R2, c2, h, p)
    Mp = orc.far_to_far(M1, c1, cp, h, p)
    Mp = orc.far_to_far(M2, c2, cp, h, p, out=Mp)
    direct = orc.farfield_moments(R, cp, h, p)
    scale = orc.farfield_moments(np.abs(R - cp) + cp, cp, h, p)  # sum of |terms|
    assert np.all(np.abs(Mp - direct) <= 1e-12 * (np.abs(scale) + 1e-300))


@pytest.mark.parametrize("D,p", [(1, 8), (2, 6), (3, 4), (4, 2)])
def test_local_to_local_is_exact(orc, D, p):
    rng = np.random.default_rng(70 + D)
    h = 0.1
    c = rng.random(D)
    c2 = c + rng.uniform(-0.05, 0.05, size=D)
    L = rng.normal(size=p ** D)
    L2 = orc.local_to_local(L, c, c2, h, p)
    q = box_points(rng, 30, c, 0.08)
    a = orc.eval_local(L, c, h, p, q)
    b = orc.eval_local(L2, c2, h, p, q)
    assert np.allclose(a, b, rtol=1e-10, atol=1e-10 * np.abs(L).sum())


def test_storage_radix_larger_than_order(orc):
    # Tables stored with radix p_max and read at a lower order agree with
    # tables stored at that order.
    rng = np.random.default_rng(80)
    D, h, p, pm = 3, 0.1, 2, 4
    c = rng.random(D)
    R = box_points(rng, 20, c, 0.05)
    q = box_points(rng, 5, c, 0.3)
    M_small = orc.farfield_moments(R, c, h, p)
    M_big = orc.farfield_moments(R, c, h, p, pm=pm)
    assert np.allclose(orc.eval_farfield(M_small, c, h, p, q),
                       orc.eval_farfield(M_big, c, h, p, q, pm=pm), rtol=1e-14)
