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


@pytest.mark.parametrize("D,side,h,efp", [(6, 0.2, 0.3, 0.0), (7, 0.2, 0.3, 0.0), (7, 1.0, 0.5, 1e-3),
                                          (8, 0.2, 0.3, 0.0), (12, 0.15, 0.3, 0.0), (16, 0.1, 0.25, 0.0),
                                          (16, 1.0, 0.5, 1e-3), (20, 0.08, 0.3, 0.0), (32, 0.05, 0.2, 0.0),
                                          (32, 1.0, 0.9, 1e-3)])
def test_whole_node_exact_sum_high_dimension(dev, orc, D, side, h, efp):
    # D >= 6: one base entry (root, root) whose expansion bound puts it in
    # the tensor-core form; each term's error is then at most eps_fp / 4
    # (plus ex2.approx's 2^-21 and the float32 summation)
    rng = np.random.default_rng(60 + D)
    X = (side * rng.random((2000, D))).astype(np.float32)
    t = dfgt.Tree(dev, to_cuda(X), eps_fp=efp)
    G = dfgt.apply_pairs(dev, t, t, [0], [0], [_lib.ACT_BASE], [1], h).cpu().numpy()
    want = orc.naive_kde(X.astype(np.float64), X.astype(np.float64), h)
    rel = np.abs(G - want) / want
    allowance = efp if efp > 0 else 2e-5
    assert rel.max() <= allowance / 4 + 2e-6, (D, rel.max())


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
