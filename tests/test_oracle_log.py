"""Pins for the oracle's log G (Eq. 5 in log-sum-exp form with a per-query
shift), the reference for sums that underflow double precision.

None of these retypes the oracle's loop: they use closed forms (one and two
reference points, coincident points as h -> 0), the factorisation of the
Gaussian over a Cartesian grid evaluated one dimension at a time with
scipy's logsumexp, agreement with the plain sum wherever that is
representable, and invariances.  Coordinates in the closed-form cases are
multiples of 1/8, so every squared distance is exact in binary.
"""
import numpy as np
import pytest
from scipy.special import logsumexp


def test_single_reference_point_far_below_double_range(orc):
    # G = exp(-|q - r|^2 / 2h^2) exactly; at D = 32, h = 0.01 that is
    # exp(-1.6e5), which no float format holds, while log G is exact.
    D = 32
    r = np.full((1, D), 0.125)
    q = np.zeros((3, D))
    q[1, :] = 1.0
    q[2, ::2] = 0.5
    for h in (0.01, 0.5):
        d2 = ((q - r) ** 2).sum(1)
        want = -d2 / (2 * h * h)
        got = orc.log_naive_kde(q, r, h)
        assert np.allclose(got, want, rtol=1e-15, atol=0)


def test_two_reference_points_closed_form(orc):
    # log(e^-a + e^-b) = -a + log(1 + e^-(b - a)) for a <= b, here with
    # a and b in the thousands (both terms underflow double)
    D = 4
    q = np.zeros((1, D))
    r1 = np.array([[0.5, 0.25, 0.0, 0.125]])
    r2 = np.array([[0.5, 0.25, 0.125, 0.125]])
    R = np.concatenate([r2, r1])  # nearer point second
    for h in (0.004, 0.01, 0.05):
        a = (r1 ** 2).sum() / (2 * h * h)
        b = (r2 ** 2).sum() / (2 * h * h)
        want = -a + np.log1p(np.exp(-(b - a)))
        got = orc.log_naive_kde(q, R, h)[0]
        assert got == pytest.approx(want, rel=1e-15, abs=0)
        if h == 0.004:
            assert np.exp(got) == 0.0  # the plain sum would be 0
    # equal distances: log 2 above the shared exponent
    R = np.array([[0.25, 0.0, 0.0, 0.0], [0.0, 0.25, 0.0, 0.0]])
    got = orc.log_naive_kde(q, R, 0.01)[0]
    assert got == pytest.approx(-0.0625 / 2e-4 + np.log(2.0), rel=1e-15)


def test_zero_bandwidth_log_counts_coincident_points(orc):
    # as h -> 0 only coincident points remain: log G -> log(count)
    rng = np.random.default_rng(3)
    base = np.round(rng.random((9, 3)) * 8) / 8 + np.arange(9)[:, None]  # points at least 1 apart
    mult = np.arange(1, 10)
    R = np.repeat(base, mult, axis=0)
    R = R[rng.permutation(len(R))]
    got = orc.log_naive_kde(base, R, 1e-3)
    assert np.allclose(got, np.log(mult), rtol=0, atol=1e-15)


@pytest.mark.parametrize("D,h", [(3, 0.002), (3, 0.05), (4, 0.004)])
def test_grid_factorisation_in_log_space(orc, D, h):
    # For R a Cartesian grid, log G(q) = sum_d log sum_i exp(-(q_d - x_{d,i})^2 / 2h^2);
    # each one-dimensional sum goes through scipy's logsumexp, so the
    # comparison holds far below the double range (h = 0.002 gives G ~ e^-900).
    rng = np.random.default_rng(40 + D)
    axes = [np.sort(rng.random(5 + d)) for d in range(D)]
    mesh = np.meshgrid(*axes, indexing="ij")
    R = np.stack([m.ravel() for m in mesh], axis=1)
    Q = rng.random((20, D))
    got = orc.log_naive_kde(Q, R, h)
    want = np.zeros(len(Q))
    for d in range(D):
        want += logsumexp(-(Q[:, d:d + 1] - axes[d][None, :]) ** 2 / (2 * h * h), axis=1)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12)
    if h == 0.002:
        assert np.all(want < -745)  # below the smallest double: only the log form holds it


def test_log_agrees_with_plain_sum_where_representable(orc):
    rng = np.random.default_rng(7)
    R = rng.random((400, 3))
    Q = rng.random((50, 3))
    for h in (0.02, 0.1, 0.7):
        G = orc.naive_kde(Q, R, h)
        L = orc.log_naive_kde(Q, R, h)
        ok = G > 1e-300
        assert ok.any()
        assert np.allclose(np.exp(L[ok]), G[ok], rtol=1e-12, atol=0)


def test_log_permutation_and_translation_invariance(orc):
    rng = np.random.default_rng(8)
    R = rng.random((300, 5))
    Q = rng.random((30, 5)) + 2.0  # far from every reference: G underflows at h = 0.01
    L = orc.log_naive_kde(Q, R, 0.01)
    assert np.all(L < -745)
    Lp = orc.log_naive_kde(Q, R[rng.permutation(300)], 0.01)
    assert np.allclose(L, Lp, rtol=1e-13)
    shift = np.array([0.25, -1.5, 3.0, 0.5, -0.125])
    Lt = orc.log_naive_kde(Q + shift, R + shift, 0.01)
    assert np.allclose(L, Lt, rtol=1e-9)
