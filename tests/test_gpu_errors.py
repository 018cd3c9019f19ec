"""Failures come back as status codes (no abort, no device fault)."""
import numpy as np
import pytest

import paper_1102_2878_gb300 as dfgt
from conftest import to_cuda

pytestmark = pytest.mark.gpu


def test_non_finite_coordinates_rejected(dev):
    x = np.random.default_rng(0).random((100, 3)).astype(np.float32)
    x[17, 1] = np.nan
    with pytest.raises(dfgt.DFGTError, match="EINVAL"):
        dfgt.Tree(dev, to_cuda(x))
    x[17, 1] = np.inf
    with pytest.raises(dfgt.DFGTError, match="EINVAL"):
        dfgt.Tree(dev, to_cuda(x))


def test_bad_arguments_rejected(dev):
    x = np.random.default_rng(1).random((100, 3)).astype(np.float32)
    t = dfgt.Tree(dev, to_cuda(x))
    for hs, eps in [([0.1], 0.0), ([0.1], 1.0), ([0.0], 1e-2), ([-1.0], 1e-2), ([np.inf], 1e-2),
                    ([0.1], 1e-6)]:
        with pytest.raises(dfgt.DFGTError, match="EINVAL"):
            dfgt.kde_sum(dev, t, t, hs, eps)
    t2 = dfgt.Tree(dev, to_cuda(x[:, :2].copy()))
    with pytest.raises(dfgt.DFGTError, match="EINVAL"):
        dfgt.kde_sum(dev, t, t2, [0.1], 1e-2)
    with pytest.raises(dfgt.DFGTError, match="EINVAL"):
        dfgt.Tree(dev, to_cuda(x), leaf_size=100000)
    with pytest.raises(dfgt.DFGTError, match="EINVAL"):
        dev.set_capacity(0, 10)
    # the context stays usable after rejected calls
    G, _ = dfgt.kde_sum(dev, t, t, [0.1], 1e-2)
    assert np.isfinite(G.cpu().numpy()).all()


def test_float_allowance_rule(dev):
    # eps_fp = 0 leaves the float allowance to each sum: 1% of eps within
    # [2e-5, 1e-4]; eps must exceed it.  An explicit eps_fp on either tree
    # takes precedence.
    x = np.random.default_rng(2).random((300, 2)).astype(np.float32)
    t = dfgt.Tree(dev, to_cuda(x))
    dfgt.kde_sum(dev, t, t, [0.1], 1e-4)       # allowance 2e-5
    with pytest.raises(dfgt.DFGTError, match="EINVAL"):
        dfgt.kde_sum(dev, t, t, [0.1], 1.5e-5)  # below the 2e-5 floor
    with pytest.raises(dfgt.DFGTError, match="EINVAL"):
        dfgt.kde_sum_loo(dev, t, [0.1], 1.5e-5)
    te = dfgt.Tree(dev, to_cuda(x), eps_fp=5e-4)
    with pytest.raises(dfgt.DFGTError, match="EINVAL"):
        dfgt.kde_sum(dev, t, te, [0.1], 4e-4)
    G, _ = dfgt.kde_sum(dev, t, te, [0.1], 1e-3)
    assert np.isfinite(G.cpu().numpy()).all()


def test_bounded_waits_report_timeout_and_context_recovers(dev):
    # Every grid barrier of the cooperative launches waits for one arrival
    # that never comes (a host-side switch, nothing faults): each block gives
    # up after its poll limit, records the timeout and returns, so the build
    # and the sum come back with DFGT_ETIMEOUT instead of hanging.
    import time

    from paper_1102_2878_gb300 import datagen

    x = datagen.anisotropic_mixture(3000, 3, 4, 1e-4, 1e-2, seed=11)
    pts = to_cuda(x)
    t = dfgt.Tree(dev, pts)
    want, _ = dfgt.kde_sum(dev, t, t, [0.02, 0.2], 1e-2)
    try:
        dev.test_wait_timeout(True)
        t0 = time.perf_counter()
        with pytest.raises(dfgt.DFGTError, match="ETIMEOUT"):
            dfgt.Tree(dev, pts)
        with pytest.raises(dfgt.DFGTError, match="ETIMEOUT"):
            dfgt.kde_sum(dev, t, t, [0.02, 0.2], 1e-2)
        assert time.perf_counter() - t0 < 30.0  # the calls came back, the waits did run out
    finally:
        dev.test_wait_timeout(False)
    # the context serves the next normal calls, with the same results
    t2 = dfgt.Tree(dev, pts)
    got, _ = dfgt.kde_sum(dev, t2, t2, [0.02, 0.2], 1e-2)
    rel = np.abs(got.cpu().numpy() - want.cpu().numpy()) / want.cpu().numpy()
    assert rel.max() <= 2e-2
    assert dfgt._lib.load().dfgt_test_wait_timeout(dev.h, 2) == 1  # DFGT_EINVAL
    t.close()
    t2.close()
