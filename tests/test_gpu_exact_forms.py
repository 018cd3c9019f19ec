"""The two forms of the exact sums (DFGTBase): a run whose expansion bound
is small enough (a quarter of the float allowance eps_fp) is summed in the
expanded form B_r + W_q . r~ about the query box centre, the others in
the direct form.  Whole-node exact sums must stay within eps_fp = 2e-5 of
the oracle's float64 sums in either form, and traversals must keep the
eps guarantee whatever share each form takes."""
import numpy as np
import pytest

import paper_1102_2878_gb300 as dfgt
from conftest import to_cuda
from paper_1102_2878_gb300 import _lib, datagen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("D,side,h", [(1, 1.0, 0.6), (2, 1.0, 0.8), (3, 1.0, 0.9), (3, 0.3, 0.5),
                                      (4, 0.5, 0.6), (5, 0.3, 0.5)])
def test_whole_node_exact_sum_within_float_allowance(dev, orc, D, side, h):
    # one base entry (root, root): 3000 queries against 3000 references in
    # one run; the span of the root box over h puts it in the expanded form
    rng = np.random.default_rng(40 + D)
    X = (side * rng.random((3000, D))).astype(np.float32)
    t = dfgt.Tree(dev, to_cuda(X))
    G = dfgt.apply_pairs(dev, t, t, [0], [0], [_lib.ACT_BASE], [1], h).cpu().numpy()
    want = orc.naive_kde(X.astype(np.float64), X.astype(np.float64), h)
    rel = np.abs(G - want) / want
    assert rel.max() <= 2e-5, (D, rel.max())
    # the same sum forced onto the direct form (float allowance too small
    # for either expanded form) agrees as well
    td = dfgt.Tree(dev, to_cuda(X), eps_fp=1e-7)
    Gd = dfgt.apply_pairs(dev, td, td, [0], [0], [_lib.ACT_BASE], [1], h).cpu().numpy()
    assert (np.abs(Gd - want) / want).max() <= 2e-5


@pytest.mark.parametrize("eps", [1e-2, 1e-3])
def test_traversal_with_both_forms(dev, orc, eps):
    x = datagen.anisotropic_mixture(20000, 3, 16, 1e-4, 1e-2, seed=5)
    hs = [0.01, 0.03, 0.1]
    t = dfgt.Tree(dev, to_cuda(x))
    G, st = dfgt.kde_sum(dev, t, t, hs, eps)
    assert 0 < st["base_expanded"] < st["base_interactions"]
    G = G.cpu().numpy()
    x64 = x.astype(np.float64)
    for i, h in enumerate(hs):
        ref = orc.naive_kde(x64, x64, h)
        rel = np.abs(G[i] - ref) / ref
        assert rel.max() <= eps, (h, rel.max())


def test_forms_partition_the_interactions(dev):
    # a tree whose float allowance rules out the expanded form (but for
    # near-degenerate query boxes) sums in the direct form, and the same
    # sums agree
    x = datagen.anisotropic_mixture(8000, 3, 8, 1e-4, 1e-2, seed=9)
    hs = [0.02, 0.08]
    t = dfgt.Tree(dev, to_cuda(x))
    G, st = dfgt.kde_sum(dev, t, t, hs, 1e-2)
    td = dfgt.Tree(dev, to_cuda(x), eps_fp=1e-7)
    Gd, std = dfgt.kde_sum(dev, td, td, hs, 1e-2)
    assert st["base_expanded"] > 0.5 * st["base_interactions"]
    assert std["base_expanded"] < 0.01 * std["base_interactions"]
    rel = (G - Gd).abs() / Gd
    assert rel.max().item() <= 2e-2


U = 2.0 ** -24


def tc_kappa(D):
    """kappa of the tensor form's bound (base_hd_forms.cuh): 26 + 4 KC, KC
    the chained K16 steps of DM = 8, 16 or 32 padded coordinates."""
    dm = 8 if D <= 8 else 16 if D <= 16 else 32
    return 26 + 4 * ((3 * dm + 2 + 15) // 16)


def tc_tolerance(X, Q, h, e1, D):
    """Relative error allowed to one query's exact sum in the tensor form:
    2^-21 (ex2) + E1 + 2 kappa u xbar (xbar the kernel-weighted mean
    exponent, natural units) + 2^-20 for the float32 summation."""
    tol = np.empty(len(Q))
    for i, q in enumerate(Q):
        x = ((X - q) ** 2).sum(1) / (2 * h * h)
        K = np.exp(-x)
        tol[i] = 2.0 ** -21 + e1 + 2 * tc_kappa(D) * U * (K * x).sum() / K.sum() + 2.0 ** -20
    return tol


@pytest.mark.parametrize("D,side,h", [(6, 0.3, 0.3), (7, 1.0, 0.6), (8, 0.3, 0.3), (12, 0.3, 0.3),
                                      (16, 0.25, 0.3), (16, 1.0, 0.9), (20, 0.2, 0.3), (32, 0.2, 0.4),
                                      (32, 1.0, 1.5)])
def test_whole_node_exact_sum_high_dimension(dev, orc, D, side, h):
    # D >= 6: one base entry (root, root) of 2000 queries against 2000
    # references in the tensor-core form (float allowance 1e-3: E1 =
    # 8 kappa u rho^2 / 2h^2 <= eps_fp / 4 for these boxes), within the
    # form's bound of the oracle's float64 sums
    rng = np.random.default_rng(60 + D)
    X = (side * rng.random((2000, D))).astype(np.float32)
    efp = 1e-3
    t = dfgt.Tree(dev, to_cuda(X), eps_fp=efp)
    G, st = dfgt.apply_pairs(dev, t, t, [0], [0], [_lib.ACT_BASE], [1], h, with_stats=True)
    assert st["base_expanded"] == st["base_interactions"] == 2000 * 2000, st
    G = G.cpu().numpy()
    X64 = X.astype(np.float64)
    want = orc.naive_kde(X64, X64, h)
    rel = np.abs(G - want) / want
    lo, hi = X.min(0).astype(np.float64), X.max(0).astype(np.float64)
    rho2 = (((hi - lo) / 2) ** 2).sum()
    e1 = 8 * tc_kappa(D) * U * rho2 / (2 * h * h)
    assert e1 <= efp / 4
    sample = rng.choice(2000, size=300, replace=False)
    tol = tc_tolerance(X64, X64[sample], h, e1, D)
    assert np.all(rel[sample] <= tol), (D, float((rel[sample] / tol).max()))
    assert rel.max() <= efp, (D, rel.max())
    # the same sum forced onto the direct form agrees within both bounds
    td = dfgt.Tree(dev, to_cuda(X), eps_fp=1e-7)
    Gd, sd = dfgt.apply_pairs(dev, td, td, [0], [0], [_lib.ACT_BASE], [1], h, with_stats=True)
    assert sd["base_expanded"] == 0
    assert (np.abs(Gd.cpu().numpy() - want) / want).max() <= efp


@pytest.mark.parametrize("D", [8, 16, 32])
def test_tensor_form_ragged_runs(dev, orc, D):
    # many base entries of one query node: reference tiles that end part
    # way (ragged 128-column tiles), query blocks past 128 rows, and runs
    # spanning several 32-entry chunks
    rng = np.random.default_rng(90 + D)
    X = (0.3 * rng.random((3001, D))).astype(np.float32)
    Y = (0.3 * rng.random((1777, D))).astype(np.float32)
    qt = dfgt.Tree(dev, to_cuda(Y), eps_fp=1e-3, leaf_size=200)
    rt = dfgt.Tree(dev, to_cuda(X), eps_fp=1e-3, leaf_size=7)
    rinfo = rt.export()
    leaves = np.flatnonzero(rinfo["left"] < 0)
    h = 0.35
    G, st = dfgt.apply_pairs(dev, qt, rt, [0] * len(leaves), list(leaves), [_lib.ACT_BASE] * len(leaves),
                             [1] * len(leaves), h, with_stats=True)
    assert st["base_expanded"] == st["base_interactions"] == 1777 * 3001, st
    want = orc.naive_kde(Y.astype(np.float64), X.astype(np.float64), h)
    rel = np.abs(G.cpu().numpy() - want) / want
    assert rel.max() <= 1e-3, rel.max()


@pytest.mark.parametrize("eps", [1e-2, 1e-3])
def test_high_dimension_traversal_with_tensor_form(dev, orc, eps):
    x = datagen.manifold_points(6000, 16, 4, 0.01, seed=12)
    hs = [0.3, 0.6, 1.0]
    t = dfgt.Tree(dev, to_cuda(x), eps_fp=2.5e-4 if eps == 1e-2 else 0.0)
    G, st = dfgt.kde_sum(dev, t, t, hs, eps)
    if eps == 1e-2:
        assert st["base_expanded"] > 0
    G = G.cpu().numpy()
    x64 = x.astype(np.float64)
    for i, h in enumerate(hs):
        ref = orc.naive_kde(x64, x64, h)
        rel = np.abs(G[i] - ref) / ref
        assert rel.max() <= eps, (h, rel.max())


def test_high_dimension_bichromatic_and_leave_one_out(dev, orc):
    # D = 8 with the tensor form engaged (eps_fp 1e-3): a separate query set
    # against the references, and leave-one-out sums over the references
    # (runs holding a self entry stay on the direct form)
    rng = np.random.default_rng(77)
    X = (0.4 * rng.random((5000, 8))).astype(np.float32)
    Qp = (0.4 * rng.random((1500, 8))).astype(np.float32)
    hs = [0.4, 0.8]
    rt = dfgt.Tree(dev, to_cuda(X), eps_fp=1e-3)
    qt = dfgt.Tree(dev, to_cuda(Qp), eps_fp=1e-3)
    G, st = dfgt.kde_sum(dev, qt, rt, hs, 1e-2)
    assert st["base_expanded"] > 0
    G = G.cpu().numpy()
    S, sl = dfgt.kde_sum_loo(dev, rt, hs, 1e-2)
    S = S.cpu().numpy()
    for i, h in enumerate(hs):
        ref = orc.naive_kde(Qp.astype(np.float64), X.astype(np.float64), h)
        assert (np.abs(G[i] - ref) / ref).max() <= 1e-2, h
        refl = orc.loo_sums(X.astype(np.float64), h)
        assert (np.abs(S[i] - refl) / refl).max() <= 1e-2, h
