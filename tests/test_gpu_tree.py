"""Device kd-tree (Algorithm 2) invariants and raw moments against the oracle."""
import numpy as np
import pytest

import paper_1102_2878_gb300 as dfgt
from conftest import to_cuda
from paper_1102_2878_gb300 import datagen

pytestmark = pytest.mark.gpu


def check_tree(x, t, leaf):
    n, D = x.shape
    perm, lo, hi = t["perm"], t["lo"], t["hi"]
    beg, cnt, left = t["begin"], t["count"], t["left"]
    nn = t["info"]["n_nodes"]
    assert np.array_equal(np.sort(perm), np.arange(n))
    assert beg[0] == 0 and cnt[0] == n
    xp = x[perm]
    for j in range(nn):
        pts = xp[beg[j]:beg[j] + cnt[j]]
        assert cnt[j] >= 1
        # tight bounding box
        assert np.array_equal(lo[j], pts.min(0)) and np.array_equal(hi[j], pts.max(0))
        if left[j] < 0:
            continue
        a, b = left[j], left[j] + 1
        # children partition the parent, adjacent, left first
        assert beg[a] == beg[j] and beg[b] == beg[a] + cnt[a] and cnt[a] + cnt[b] == cnt[j]
        assert cnt[a] > 0 and cnt[b] > 0
        # widest dimension split at the float32 midpoint
        ext = hi[j] - lo[j]
        sd = int(np.argmax(ext))
        sc = np.float32(0.5) * (lo[j][sd] + hi[j][sd])
        assert np.all(xp[beg[a]:beg[a] + cnt[a], sd] <= sc)
        assert np.all(xp[beg[b]:beg[b] + cnt[b], sd] > sc)
        assert cnt[j] > leaf
    leaves = np.where(left < 0)[0]
    assert cnt[leaves].sum() == n
    # the node's ball about the float box centre holds every point of it, and
    # is no wider than the box's half diagonal allows (plus float rounding)
    rad = t["radius"].astype(np.float64)
    for j in range(nn):
        pts = xp[beg[j]:beg[j] + cnt[j]].astype(np.float64)
        c = (np.float32(0.5) * (lo[j] + hi[j])).astype(np.float64)
        dmax = np.sqrt(((pts - c) ** 2).sum(1).max())
        assert dmax <= rad[j], (j, dmax, rad[j])
        half_diag = np.sqrt((np.maximum(hi[j] - c, c - lo[j]) ** 2).sum())
        # (float32 squares of sides below 1e-19 are subnormal: an absolute slack)
        assert rad[j] <= half_diag * (1 + 1e-5) + 1e-20, (j, rad[j], half_diag)


@pytest.mark.parametrize("D,n,leaf", [(1, 1000, 8), (2, 5000, 32), (3, 20011, 32), (5, 3000, 16),
                                      (8, 2000, 32), (16, 1500, 64), (2, 400003, 128)])
def test_tree_invariants(dev, D, n, leaf):
    x = datagen.isotropic_mixture(n, D, 6, 0.05, seed=D + n)
    tree = dfgt.Tree(dev, to_cuda(x), leaf_size=leaf)
    t = tree.export()
    check_tree(x, t, leaf)
    # leaves hold at most `leaf` points unless their points coincide
    left, cnt, lo, hi = t["left"], t["count"], t["lo"], t["hi"]
    for j in np.where(left < 0)[0]:
        assert cnt[j] <= leaf or np.all(lo[j] == hi[j])


def test_tree_degenerate_points(dev):
    x = np.tile(np.float32([[0.25, 0.5, 0.75]]), (300, 1))
    x[:100, 0] = 0.3  # two distinct positions
    t = dfgt.Tree(dev, to_cuda(x), leaf_size=8).export()
    check_tree(x, t, 8)
    assert t["info"]["n_leaves"] == 2


def test_tree_single_point(dev):
    t = dfgt.Tree(dev, to_cuda(np.float32([[0.1, 0.2]])), leaf_size=4).export()
    assert t["info"]["n_nodes"] == 1 and t["count"][0] == 1


@pytest.mark.parametrize("D", [1, 2, 3, 4, 5])
def test_raw_moments_match_oracle(dev, orc, D):
    # raw moments sum (r-c)^alpha/alpha! are the oracle's moments at h = 1/sqrt(2)
    x = datagen.isotropic_mixture(3000, D, 4, 0.1, seed=40 + D)
    tree = dfgt.Tree(dev, to_cuda(x), leaf_size=16)
    t = tree.export()
    pm = t["info"]["p_max"]
    xp = x.astype(np.float64)[t["perm"]]
    h = 1.0 / np.sqrt(2.0)
    rng = np.random.default_rng(D)
    nodes = np.concatenate([[0], rng.choice(t["info"]["n_nodes"], size=40, replace=False)])
    for j in nodes:
        pts = xp[t["begin"][j]:t["begin"][j] + t["count"][j]]
        c = 0.5 * (t["lo"][j].astype(np.float64) + t["hi"][j].astype(np.float64))
        want = orc.farfield_moments(pts, c, h, pm)
        scale = orc.farfield_moments(np.abs(pts - c) + c, c, h, pm)
        assert np.all(np.abs(t["moments"][j] - want) <= 1e-10 * scale + 1e-300), j


def test_node_buffer_growth(orc):
    # points 1.5^-k: every midpoint split peels off one or two points, so the
    # tree has far more nodes than the 4n/leaf + 16 first reserved and the
    # build's node buffer grows (a fresh context starts with none)
    ctx = dfgt.Context(0)
    x = (1.5 ** -np.arange(200, dtype=np.float64)).astype(np.float32)[:, None]
    tree = dfgt.Tree(ctx, to_cuda(x), leaf_size=8)
    t = tree.export()
    assert t["info"]["n_nodes"] > 4 * 200 // 8 + 16
    check_tree(x, t, 8)
    hs = np.array([0.01, 0.3])
    G, _ = dfgt.kde_sum(ctx, tree, tree, hs, 1e-3)
    G = G.cpu().numpy()
    for i, h in enumerate(hs):
        ref = orc.naive_kde(x.astype(np.float64), x.astype(np.float64), h)
        assert np.all(np.abs(G[i] - ref) <= 1e-3 * ref)


def test_tree_arenas_reused():
    # trees come from one pool per context: a freed tree's memory serves the
    # next build, and live trees are never disturbed by it
    ctx = dfgt.Context(0)
    xa = datagen.isotropic_mixture(5000, 3, 5, 0.05, seed=1)
    a = dfgt.Tree(ctx, to_cuda(xa), leaf_size=16)
    ea = a.export()
    for k, n in enumerate([3000, 7000, 1000, 7000]):
        x = datagen.isotropic_mixture(n, 3, 5, 0.05, seed=10 + k)
        b = dfgt.Tree(ctx, to_cuda(x), leaf_size=16)
        check_tree(x, b.export(), 16)
        b.close()
    ea2 = a.export()
    for key in ("perm", "lo", "hi", "begin", "count", "left", "moments"):
        assert np.array_equal(ea[key], ea2[key]), key


def test_tree_outlives_context():
    ctx = dfgt.Context(0)
    x = datagen.isotropic_mixture(2000, 2, 3, 0.1, seed=5)
    t = dfgt.Tree(ctx, to_cuda(x), leaf_size=16)
    ctx.close()
    t.close()  # the arena goes back to the pool, which then goes away
    ctx2 = dfgt.Context(0)
    check_tree(x, dfgt.Tree(ctx2, to_cuda(x), leaf_size=16).export(), 16)
