"""Randomised parity sweep: seeded random configurations (dimension, size,
leaf size, data shape, bandwidths, eps, separate or shared query set)
through the whole path, each sum held to its guarantee against the
oracle's exact float64 sums, and the leave-one-out sums of the same
points against the oracle's leave-one-out sums."""
import numpy as np
import pytest

import paper_1102_2878_gb300 as dfgt
from conftest import to_cuda
from paper_1102_2878_gb300 import datagen

pytestmark = pytest.mark.gpu

TINY = 1e-30  # sums below float32 range are outside the guarantee


def config(k):
    rng = np.random.default_rng(9000 + k)
    D = int(rng.choice([1, 2, 3, 4, 5, 7, 12]))
    n = int(rng.integers(300, 8000))
    leaf = int(rng.choice([0, 8, 32, 128]))
    eps = float(rng.choice([1e-1, 1e-2, 1e-3]))
    hs = np.sort(np.exp(rng.uniform(np.log(2e-3), np.log(1.0), size=int(rng.integers(1, 5)))))
    shape = int(rng.integers(0, 4))
    if shape == 0:
        x = datagen.isotropic_mixture(n, D, int(rng.integers(1, 9)), float(rng.uniform(0.01, 0.1)), seed=k)
    elif shape == 1:
        x = datagen.anisotropic_mixture(n, D, int(rng.integers(1, 9)), 1e-4, 1e-2, seed=k)
    elif shape == 2:
        x = rng.random((n, D)).astype(np.float32)
    else:  # clustered with exact duplicates
        base = datagen.isotropic_mixture(n // 3 + 1, D, 3, 0.05, seed=k)
        x = np.concatenate([base, base, base])[:n]
    x = np.ascontiguousarray(x.astype(np.float32))
    q = None
    if rng.random() < 0.4:  # a separate query set
        q = np.ascontiguousarray(rng.random((int(rng.integers(100, 3000)), D)).astype(np.float32))
    return D, x, q, leaf, eps, hs


@pytest.mark.parametrize("k", range(24))
def test_random_configuration(dev, orc, k):
    D, x, q, leaf, eps, hs = config(k)
    rtree = dfgt.Tree(dev, to_cuda(x), leaf_size=leaf)
    qtree = rtree if q is None else dfgt.Tree(dev, to_cuda(q), leaf_size=leaf)
    G, L, _ = dfgt.kde_sum_log(dev, qtree, rtree, hs, eps)
    G, L = G.cpu().numpy(), L.cpu().numpy()
    qx = (x if q is None else q).astype(np.float64)
    for i, h in enumerate(hs):
        # every query, in log form (Definition 1.2 for sums below any float range too)
        ref_log = orc.log_naive_kde(qx, x.astype(np.float64), h)
        err = np.abs(np.expm1(L[i] - ref_log))
        assert err.max(initial=0.0) <= eps, (k, D, len(x), leaf, eps, h, float(err.max(initial=0.0)))
        ref = np.exp(ref_log)
        ok = ref > 1e-300
        rel = np.abs(G[i][ok] - ref[ok]) / ref[ok]
        assert rel.max(initial=0.0) <= eps, (k, D, len(x), leaf, eps, h, float(rel.max(initial=0.0)))
        assert np.all(np.isfinite(G[i])) and np.all(np.isfinite(L[i]))
    if q is None and len(x) >= 2:
        S, _ = dfgt.kde_sum_loo(dev, rtree, hs, eps)
        S = S.cpu().numpy()
        for i, h in enumerate(hs):
            ref = orc.loo_sums(x.astype(np.float64), h)
            ok = ref > TINY
            rel = np.abs(S[i][ok] - ref[ok]) / ref[ok]
            assert rel.max(initial=0.0) <= eps, (k, "loo", D, len(x), leaf, eps, h, float(rel.max(initial=0.0)))
