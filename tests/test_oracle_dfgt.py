"""Pins for the oracle's dual-tree traversal (DFGTMain, Section 3.6).

The traversal is an approximation, so it is pinned by the paper's three
theorems against the exact sum: the per-query bounds bracket the exact
value (Theorem 3.1), every query accounts for every reference point once
(Theorem 3.2), and every query is within the relative tolerance
(Theorem 3.3, Definition 1.2).
"""
import numpy as np
import pytest

from paper_1102_2878_gb300 import datagen


def _points(D, n, seed):
    return datagen.isotropic_mixture(n, D, 6, 0.05, seed=seed).astype(np.float64)


CASES = [(D, h, eps) for D in (1, 2, 3, 5) for h in (0.004, 0.03, 0.2, 1.5) for eps in (1e-2, 1e-3)]


@pytest.mark.parametrize("D,h,eps", CASES)
def test_relative_error_guarantee(orc, D, h, eps):
    X = _points(D, 1500, seed=100 + D)
    G = orc.naive_kde(X, X, h)
    out = orc.dfgt(X, X, h, eps, leaf=16, want_bounds=True, want_acct=True)
    rel = np.abs(out["G"] - G) / G
    assert rel.max() <= eps
    assert np.all(out["acct"] == len(X))
    assert np.all(out["Gl"] <= G * (1 + 1e-12))
    assert np.all(out["Gu"] >= G * (1 - 1e-12))


def test_bichromatic_and_ragged_leaves(orc):
    rng = np.random.default_rng(9)
    R = _points(3, 2001, seed=11)
    Q = rng.random((333, 3))
    for h in (0.01, 0.1, 0.5):
        G = orc.naive_kde(Q, R, h)
        out = orc.dfgt(Q, R, h, 1e-2, leaf=7, want_acct=True)
        assert np.all(np.abs(out["G"] - G) <= 1e-2 * G)
        assert np.all(out["acct"] == len(R))


def test_tiny_tolerance_is_exact(orc):
    X = _points(2, 800, seed=12)
    G = orc.naive_kde(X, X, 0.05)
    out = orc.dfgt(X, X, 0.05, 1e-13, leaf=8)
    assert np.allclose(out["G"], G, rtol=1e-11)


def test_expansions_are_exercised(orc):
    # At a bandwidth comparable to the clusters the traversal uses far-field,
    # local and prune summaries, not only base cases.
    X = _points(3, 3000, seed=13)
    out = orc.dfgt(X, X, 0.5, 1e-2, leaf=16)
    prune, F, Dl, T, base, calls = out["stats"]
    assert F > 0 and Dl > 0
    out = orc.dfgt(X, X, 0.003, 1e-2, leaf=16)
    assert out["stats"][0] > 0


def test_degenerate_inputs(orc):
    # all points coincide -> one leaf; a single point; duplicated points
    X = np.tile([[0.3, 0.7]], (50, 1))
    out = orc.dfgt(X, X, 0.1, 1e-2, leaf=4)
    assert np.allclose(out["G"], 50.0)
    one = np.array([[0.5, 0.5, 0.5]])
    assert orc.dfgt(one, one, 0.1, 1e-2)["G"][0] == pytest.approx(1.0)
    with pytest.raises(ValueError):
        orc.dfgt(one, one, -1.0, 1e-2)
