"""The dual-tree sum on the GPU against the exact FP64 oracle: every query
within eps relative (Definition 1.2, Theorem 3.3), at sizes the oracle
finishes in seconds, across dimensions, bandwidths, tolerances, leaf sizes
and the degenerate cases."""
import numpy as np
import pytest

import paper_1102_2878_gb300 as dfgt
from conftest import to_cuda
from paper_1102_2878_gb300 import datagen

pytestmark = pytest.mark.gpu


def check_eps(G, ref, eps):
    rel = np.abs(G - ref) / ref
    assert rel.max() <= eps, f"max rel err {rel.max():.3e} > eps {eps}"
    return rel.max()


@pytest.mark.parametrize("D", [1, 2, 3, 4, 5, 6, 8])
@pytest.mark.parametrize("eps", [1e-2, 1e-3])
def test_eps_guarantee_bandwidth_sweep(dev, orc, D, eps):
    x = datagen.isotropic_mixture(6000 + 13 * D, D, 6, 0.05, seed=500 + D)
    hs = list(datagen.logspace_bandwidths(0.002, 2.0, 7))
    tree = dfgt.Tree(dev, to_cuda(x))
    G, st = dfgt.kde_sum(dev, tree, tree, hs, eps)
    G = G.cpu().numpy()
    x64 = x.astype(np.float64)
    for i, h in enumerate(hs):
        check_eps(G[i], orc.naive_kde(x64, x64, h), eps)


def test_config_d2_n1e4(dev, orc):
    """D=2, N=1e4, 8 isotropic components (sigma 0.05), h=0.02, eps=1e-2: all queries."""
    x, hs, eps = datagen.workload("kde2d_n1e4")
    tree = dfgt.Tree(dev, to_cuda(x))
    G, st = dfgt.kde_sum(dev, tree, tree, hs, eps)
    x64 = x.astype(np.float64)
    check_eps(G.cpu().numpy()[0], orc.naive_kde(x64, x64, hs[0]), eps)
    assert st["n_prune"] + st["n_base"] > 0


@pytest.mark.parametrize("leaf", [1, 8, 64, 256])
def test_leaf_sizes(dev, orc, leaf):
    x = datagen.anisotropic_mixture(5000, 3, 8, 1e-4, 1e-2, seed=11)
    hs = [0.003, 0.03, 0.3]
    tree = dfgt.Tree(dev, to_cuda(x), leaf_size=leaf)
    G, _ = dfgt.kde_sum(dev, tree, tree, hs, 1e-2)
    G = G.cpu().numpy()
    x64 = x.astype(np.float64)
    for i, h in enumerate(hs):
        check_eps(G[i], orc.naive_kde(x64, x64, h), 1e-2)


@pytest.mark.parametrize("D", [2, 3, 5])
def test_bichromatic(dev, orc, D):
    r = datagen.isotropic_mixture(7001, D, 6, 0.05, seed=600 + D)
    q = datagen.isotropic_mixture(3333, D, 6, 0.05, seed=700 + D)
    hs = [0.01, 0.05, 0.3]
    qt, rt = dfgt.Tree(dev, to_cuda(q)), dfgt.Tree(dev, to_cuda(r), leaf_size=16)
    G, L, _ = dfgt.kde_sum_log(dev, qt, rt, hs, 1e-2)
    G, L = G.cpu().numpy(), L.cpu().numpy()
    for i, h in enumerate(hs):
        # every query, in log form (the sums of far queries lie below float range)
        ref_log = orc.log_naive_kde(q.astype(np.float64), r.astype(np.float64), h)
        assert np.abs(np.expm1(L[i] - ref_log)).max() <= 1e-2
        ref = np.exp(ref_log)
        ok = ref > 1e-300
        rel = np.abs(G[i][ok] - ref[ok]) / ref[ok]
        assert rel.max() <= 1e-2


def test_each_reference_counted_once(dev):
    """Theorem 3.2: with every kernel value 1 (h huge) the sum is |R| exactly."""
    r = datagen.isotropic_mixture(5000, 3, 6, 0.05, seed=1)
    q = datagen.isotropic_mixture(999, 3, 6, 0.05, seed=2)
    qt, rt = dfgt.Tree(dev, to_cuda(q), leaf_size=8), dfgt.Tree(dev, to_cuda(r), leaf_size=8)
    G, _ = dfgt.kde_sum(dev, qt, rt, [1e6], 1e-2)
    # summaries and exact sums carry float32 rounding; a reference point
    # counted twice or missed would be off by 1/5000
    assert np.allclose(G.cpu().numpy(), 5000.0, rtol=1e-6, atol=0)


def test_degenerate_inputs(dev, orc):
    # coincident points, a single point, two points
    x = np.tile(np.float32([[0.5, 0.5, 0.5]]), (500, 1))
    t = dfgt.Tree(dev, to_cuda(x), leaf_size=8)
    G, _ = dfgt.kde_sum(dev, t, t, [0.01, 1.0], 1e-2)
    assert np.allclose(G.cpu().numpy(), 500.0, rtol=1e-6)
    one = np.float32([[0.1, 0.9]])
    t1 = dfgt.Tree(dev, to_cuda(one))
    G, _ = dfgt.kde_sum(dev, t1, t1, [0.1], 1e-2)
    assert G.cpu().numpy()[0, 0] == pytest.approx(1.0, rel=1e-6)
    two = np.float32([[0.0], [1.0]])
    t2 = dfgt.Tree(dev, to_cuda(two), leaf_size=1)
    G, _ = dfgt.kde_sum(dev, t2, t2, [0.5], 1e-3)
    want = orc.naive_kde(two.astype(np.float64), two.astype(np.float64), 0.5)
    assert np.allclose(G.cpu().numpy()[0], want, rtol=1e-3)


def test_repeatable_and_batched_equals_single(dev):
    x = datagen.anisotropic_mixture(20000, 3, 16, 1e-4, 1e-2, seed=5)
    hs = [0.002, 0.02, 0.2]
    t = dfgt.Tree(dev, to_cuda(x))
    G1, s1 = dfgt.kde_sum(dev, t, t, hs, 1e-2)
    G2, s2 = dfgt.kde_sum(dev, t, t, hs, 1e-2)
    # decisions are deterministic (fixed-point bounds, so the same pairs are
    # pruned, summarised and summed); the order in which float32 partial
    # sums meet varies with atomics, so values agree to float32 rounding
    assert s1["n_base"] == s2["n_base"] and s1["n_prune"] == s2["n_prune"]
    assert s1["n_farfield"] == s2["n_farfield"] and s1["n_local"] == s2["n_local"]
    assert np.allclose(G1.cpu().numpy(), G2.cpu().numpy(), rtol=2e-6, atol=0)
    for i, h in enumerate(hs):
        Gi, _ = dfgt.kde_sum(dev, t, t, [h], 1e-2)
        assert np.allclose(Gi.cpu().numpy()[0], G1.cpu().numpy()[i], rtol=2e-6, atol=0)


def test_small_work_lists_are_drained_early(dev, orc):
    x = datagen.anisotropic_mixture(8000, 3, 8, 1e-4, 1e-2, seed=9)
    t = dfgt.Tree(dev, to_cuda(x), leaf_size=16)
    dev.set_capacity(64, 64)
    G, st = dfgt.kde_sum(dev, t, t, [0.01, 0.1], 1e-2)
    assert st["list_flushes"] > 0
    x64 = x.astype(np.float64)
    for i, h in enumerate([0.01, 0.1]):
        check_eps(G.cpu().numpy()[i], orc.naive_kde(x64, x64, h), 1e-2)


def test_host_buffer_entry_matches_device_entry(dev):
    x = datagen.anisotropic_mixture(10000, 3, 8, 1e-4, 1e-2, seed=21)
    hs = [0.005, 0.05]
    t = dfgt.Tree(dev, to_cuda(x))
    Gd, _ = dfgt.kde_sum(dev, t, t, hs, 1e-2)
    Gh, st = dfgt.kde_host(dev, x, None, hs, 1e-2)
    assert np.allclose(Gh, Gd.cpu().numpy(), rtol=2e-6)


def test_dfgt_against_gpu_bruteforce(dev):
    x = datagen.anisotropic_mixture(50000, 3, 32, 1e-4, 1e-2, seed=2)
    hs = list(datagen.logspace_bandwidths(1e-3, 1.0, 10))
    t = dfgt.Tree(dev, to_cuda(x))
    G, st = dfgt.kde_sum(dev, t, t, hs, 1e-2)
    Gb = dfgt.kde_sum_bruteforce(dev, to_cuda(x), to_cuda(x), hs)
    rel = ((G - Gb).abs() / Gb).max().item()
    assert rel <= 1e-2 + 1e-5


def test_autotune_picks_a_candidate_and_stays_exact(dev, orc):
    # the autotuner returns one of its candidates, and a tree built with the
    # chosen options gives sums within eps
    x, hs, eps = datagen.workload("kde2d_n1e4")
    pts = to_cuda(x)
    opts, ms = dfgt.autotune(dev, pts, hs, eps, trials=1)
    assert opts["leaf_size"] in (32, 64, 96, 128, 160, 192)
    assert opts["base_block"] in (2048, 4096, 8192)
    assert opts["p_max"] in (6, 5)  # D = 2: the paper's p_max = 6, or one below it
    assert ms > 0
    t = dfgt.Tree(dev, pts, leaf_size=opts["leaf_size"], base_block=opts["base_block"], p_max=opts["p_max"])
    G, _ = dfgt.kde_sum(dev, t, t, hs, eps)
    ref = orc.naive_kde(x.astype(np.float64), x.astype(np.float64), hs[0])
    assert np.all(np.abs(G.cpu().numpy()[0] - ref) <= eps * ref)


def test_autotune_keeps_a_fixed_order_and_each_order_stays_exact(dev, orc):
    # a caller's p_max is kept; every order the search tries keeps eps
    x, hs, eps = datagen.workload("kde2d_n1e4")
    pts = to_cuda(x)
    opts, _ = dfgt.autotune(dev, pts, hs, eps, trials=1, p_max=4)
    assert opts["p_max"] == 4
    ref = orc.naive_kde(x.astype(np.float64), x.astype(np.float64), hs[0])
    for p in (6, 5, 4):
        t = dfgt.Tree(dev, pts, p_max=p)
        G, st = dfgt.kde_sum(dev, t, t, hs, eps)
        assert np.all(np.abs(G.cpu().numpy()[0] - ref) <= eps * ref), p


def test_query_batches_match_single_calls(dev, orc):
    # batches grouped into query trees (one per batch here) give every query's
    # log-form sum within eps of the oracle's log G, underflowing sums included
    refs, batches, hs, _ = datagen.bichromatic("kde32d_r1e6_q64batches", nr=20_000, nbatch=4, batch_hi=4_000)
    rt = dfgt.Tree(dev, to_cuda(refs), eps_fp=5e-4)
    eps = 1e-2
    sizes = [len(b) for b in batches]
    outs, st = dfgt.kde_sum_batches(dev, [to_cuda(b) for b in batches], rt, hs[::4], eps, eps_fp=5e-4,
                                    max_queries=max(sizes) + 1, log=True)
    assert len(outs) == len(batches) and st["rounds"] > 0
    r64 = refs.astype(np.float64)
    rng = np.random.default_rng(7)
    for b, (G, L) in zip(batches, outs):
        assert G.shape == L.shape == (len(hs[::4]), len(b))
        L = L.cpu().numpy()
        pick = rng.choice(len(b), size=min(len(b), 64), replace=False)
        for i, h in enumerate(hs[::4]):
            ref = orc.log_naive_kde(b.astype(np.float64)[pick], r64, h)
            assert np.all(np.abs(np.expm1(L[i][pick] - ref)) <= eps), h
