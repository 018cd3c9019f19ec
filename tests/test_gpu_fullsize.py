"""Full-size workloads in the benchmark's launch configuration.

The oracle cannot sum every query at these sizes, so it checks a seeded
sample of queries one by one against the full reference set; the GPU
brute force (itself checked against the oracle on the sample, 1e-5)
covers every query, and the dual-tree result must be within eps of it
everywhere.
"""
import numpy as np
import pytest

import paper_1102_2878_gb300 as dfgt
from conftest import to_cuda
from paper_1102_2878_gb300 import datagen

pytestmark = pytest.mark.gpu


def run_workload(dev, orc, name, nsample, n=None):
    x, hs, eps = datagen.workload(name, n)
    pts = to_cuda(x)
    t = dfgt.Tree(dev, pts)
    G, st = dfgt.kde_sum(dev, t, t, hs, eps)
    Gb = dfgt.kde_sum_bruteforce(dev, pts, pts, hs)
    G, Gb = G.cpu().numpy(), Gb.cpu().numpy()
    rng = np.random.default_rng(12345)
    sample = rng.choice(len(x), size=nsample, replace=False)
    x64 = x.astype(np.float64)
    for i, h in enumerate(hs):
        ref = orc.naive_kde(x64[sample], x64, h)
        assert np.all(np.abs(Gb[i][sample] - ref) <= 1e-5 * ref), (name, h)
        rel = np.abs(G[i][sample] - ref) / ref
        assert rel.max() <= eps, (name, h, rel.max())
        # every query against the (checked) brute force
        relb = np.abs(G[i] - Gb[i]) / Gb[i]
        assert relb.max() <= eps + 1e-5, (name, h, relb.max())
    return st


def test_kde3d_n2e5_sweep10(dev, orc):
    st = run_workload(dev, orc, "kde3d_n2e5_sweep10", 200)
    assert st["rounds"] > 0


def test_kde5d_n5e5(dev, orc):
    run_workload(dev, orc, "kde5d_n5e5", 64)


def test_kde16d_manifold(dev, orc):
    run_workload(dev, orc, "kde16d_n1e6_sweep8", 24, n=200_000)
