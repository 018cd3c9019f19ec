"""GPU brute-force sums (Algorithm 1) against the FP64 oracle, element by
element, within 1e-5 relative."""
import numpy as np
import pytest

import paper_1102_2878_gb300 as dfgt
from conftest import to_cuda
from paper_1102_2878_gb300 import datagen

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.mark.parametrize("D", [1, 2, 3, 4, 5, 8, 16, 32])
def test_bruteforce_matches_oracle(dev, orc, D):
    # ragged sizes: not a multiple of the 128-wide tiles or of 32-reference runs
    q = datagen.isotropic_mixture(1000 + 37, D, 5, 0.08, seed=D)
    r = datagen.isotropic_mixture(2000 + 91, D, 5, 0.08, seed=100 + D)
    hs = [0.02, 0.1, 0.4] if D <= 5 else [0.2, 0.5, 1.0]
    G = dfgt.kde_sum_bruteforce(dev, to_cuda(q), to_cuda(r), hs).cpu().numpy()
    for i, h in enumerate(hs):
        ref = orc.naive_kde(q.astype(np.float64), r.astype(np.float64), h)
        mask = ref > 1e-30
        assert np.all(np.abs(G[i][mask] - ref[mask]) <= TOL * ref[mask]), (D, h)


@pytest.mark.parametrize("nh", [1, 2, 3, 7, 10, 16, 17, 33])
def test_bruteforce_bandwidth_chunks(dev, orc, nh):
    x = datagen.isotropic_mixture(777, 3, 4, 0.05, seed=3)
    hs = list(datagen.logspace_bandwidths(0.003, 2.0, nh))
    G = dfgt.kde_sum_bruteforce(dev, to_cuda(x), to_cuda(x), hs).cpu().numpy()
    x64 = x.astype(np.float64)
    for i, h in enumerate(hs):
        ref = orc.naive_kde(x64, x64, h)
        assert np.allclose(G[i], ref, rtol=TOL, atol=0), (nh, i)


def test_bruteforce_edge_sizes(dev, orc):
    rng = np.random.default_rng(0)
    for nq, nr in [(1, 1), (1, 300), (300, 1), (129, 129), (31, 33)]:
        q = rng.random((nq, 2)).astype(np.float32)
        r = rng.random((nr, 2)).astype(np.float32)
        G = dfgt.kde_sum_bruteforce(dev, to_cuda(q), to_cuda(r), [0.3]).cpu().numpy()
        ref = orc.naive_kde(q.astype(np.float64), r.astype(np.float64), 0.3)
        assert np.allclose(G[0], ref, rtol=TOL, atol=0)


@pytest.mark.parametrize("nq,nr,D", [(1, 50_000, 3), (257, 70_001, 3), (100, 9_999, 5), (64, 20_000, 8)])
def test_bruteforce_small_query_batch_split_over_references(dev, orc, nq, nr, D):
    # a query batch too small to fill the GPU splits the references into
    # slices whose partial sums are added afterwards
    q = datagen.isotropic_mixture(nq, D, 4, 0.1, seed=nq)
    r = datagen.isotropic_mixture(nr, D, 4, 0.1, seed=nr)
    hs = list(datagen.logspace_bandwidths(0.02, 0.5, 10))
    G = dfgt.kde_sum_bruteforce(dev, to_cuda(q), to_cuda(r), hs).cpu().numpy()
    for i, h in enumerate(hs):
        ref = orc.naive_kde(q.astype(np.float64), r.astype(np.float64), h)
        ok = ref > 1e-30
        assert np.all(np.abs(G[i][ok] - ref[ok]) <= TOL * ref[ok]), (nq, nr, D, h)
