"""Pins for the oracle's exact Gaussian sum (Eq. 5 / Algorithm 1).

None of these retypes the sum: they use special cases with closed forms,
limits, the factorisation of the Gaussian over a Cartesian grid, and
invariances.
"""
import math

import numpy as np
import pytest


def test_single_reference_point(orc):
    rng = np.random.default_rng(1)
    for D in (1, 2, 3, 5, 16):
        r = rng.random((1, D))
        q = rng.random((7, D))
        h = 0.3
        G = orc.naive_kde(q, r, h)
        dist2 = ((q - r) ** 2).sum(1)
        assert np.allclose(G, np.exp(-dist2 / (2 * h * h)), rtol=1e-14, atol=0)


def test_infinite_bandwidth_counts_all_points(orc):
    rng = np.random.default_rng(2)
    R = rng.random((333, 3))
    Q = rng.random((20, 3))
    G = orc.naive_kde(Q, R, 1e9)
    assert np.allclose(G, 333.0, rtol=1e-14)


def test_zero_bandwidth_counts_coincident_points(orc):
    rng = np.random.default_rng(3)
    base = rng.random((10, 2))
    mult = np.arange(1, 11)
    R = np.repeat(base, mult, axis=0)
    R = R[rng.permutation(len(R))]
    G = orc.naive_kde(base, R, 1e-30)
    assert np.array_equal(G, mult.astype(float))


@pytest.mark.parametrize("D,h", [(2, 0.05), (3, 0.2), (3, 0.01), (4, 0.1)])
def test_grid_factorisation(orc, D, h):
    # For R a Cartesian grid, the Gaussian factorises over dimensions:
    # G(q) = prod_d sum_i exp(-(q_d - x_{d,i})^2 / 2h^2).
    rng = np.random.default_rng(4 + D)
    axes = [np.sort(rng.random(6 + d)) for d in range(D)]
    mesh = np.meshgrid(*axes, indexing="ij")
    R = np.stack([m.ravel() for m in mesh], axis=1)
    Q = rng.random((25, D))
    G = orc.naive_kde(Q, R, h)
    want = np.ones(len(Q))
    for d in range(D):
        want *= np.exp(-(Q[:, d:d + 1] - axes[d][None, :]) ** 2 / (2 * h * h)).sum(1)
    assert np.allclose(G, want, rtol=1e-12, atol=1e-300)


def test_permutation_and_translation_invariance(orc):
    rng = np.random.default_rng(6)
    R = rng.random((500, 3))
    Q = rng.random((40, 3))
    G = orc.naive_kde(Q, R, 0.1)
    Gp = orc.naive_kde(Q, R[rng.permutation(500)], 0.1)
    assert np.allclose(G, Gp, rtol=1e-13)
    shift = np.array([0.25, -1.5, 3.0])
    Gt = orc.naive_kde(Q + shift, R + shift, 0.1)
    assert np.allclose(G, Gt, rtol=1e-11)
    # Queries are independent of each other.
    G1 = orc.naive_kde(Q[5:6], R, 0.1)
    assert G1[0] == G[5]
