"""Bichromatic D=32 workload: a reference set and uneven query batches
drawn separately from one 128-component mixture, 16 bandwidths, eps 1e-2
and 1e-3 (a smaller case of kde32d_r1e6_q64batches: 1e5 references, six
batches of 1e3..2e4 queries).

Each batch is summed against one reference tree with dfgt_sum_log.  Every
sampled query must meet Definition 1.2 against the FP64 oracle in log form,
|exp(log G~ - log G) - 1| <= eps, at every bandwidth, including the many
queries whose sum lies far below the float32 (and float64) range at the
small bandwidths.  The GPU brute force covers every query and is checked
against the oracle on the same sample wherever its float32 terms can hold
the sum (G >= 1e-30).

Float32 tolerance.  A term exp(-x) computed in float32 from D coordinate
differences carries at most (D+4) u x of relative error (u = 2^-24), so at
D = 32, where these sums are made of terms with x of 30..60, the brute
force is checked against sum_r K_r (2^-21 + (D+4) u x_r) + 2^-20 G, and the
dual-tree trees reserve eps_fp = 5e-4 of eps for float32 rounding (enough
for a kernel-weighted mean exponent up to ~115).
"""
import numpy as np
import pytest

import paper_1102_2878_gb300 as dfgt
from conftest import to_cuda
from paper_1102_2878_gb300 import datagen

pytestmark = pytest.mark.gpu
TINY = 1e-30
U = 2.0 ** -24
EPS_FP = 5e-4


def bruteforce_tolerance(q64, r64, h):
    """Float32 rounding bound of the exact sums of q64 against r64."""
    D = q64.shape[1]
    tol = np.zeros(len(q64))
    G = np.zeros(len(q64))
    for i, q in enumerate(q64):
        x = ((r64 - q) ** 2).sum(1) / (2 * h * h)
        K = np.exp(-x)
        tol[i] = (K * (2.0 ** -21 + (D + 4) * U * x)).sum()
        G[i] = K.sum()
    return tol + 2.0 ** -20 * G


@pytest.fixture(scope="module")
def case():
    return datagen.bichromatic("kde32d_r1e6_q64batches", nr=100_000, nbatch=6, batch_hi=20_000)


@pytest.mark.parametrize("eps_index", [0, 1])
def test_kde32d_bichromatic_batches(dev, orc, case, eps_index):
    refs, batches, hs, eps_list = case
    eps = eps_list[eps_index]
    rt = dfgt.Tree(dev, to_cuda(refs), eps_fp=EPS_FP)
    r64 = refs.astype(np.float64)
    rng = np.random.default_rng(7 + eps_index)
    checked = underflow = 0
    for bi, qx in enumerate(batches[: 6 if eps_index == 0 else 3]):
        qt = dfgt.Tree(dev, to_cuda(qx), eps_fp=EPS_FP)
        G, L, st = dfgt.kde_sum_log(dev, qt, rt, hs, eps)
        Gb = dfgt.kde_sum_bruteforce(dev, to_cuda(qx), to_cuda(refs), hs)
        G, L, Gb = G.cpu().numpy(), L.cpu().numpy(), Gb.cpu().numpy()
        sample = rng.choice(len(qx), size=min(len(qx), 32), replace=False)
        q64 = qx.astype(np.float64)[sample]
        for i, h in enumerate(hs):
            ref_log = orc.log_naive_kde(q64, r64, h)
            err = np.abs(np.expm1(L[i][sample] - ref_log))
            assert np.all(err <= eps), (bi, h, float(err.max()))
            # G~ = exp(log G~) in float64 wherever G is a normal float64
            ref = np.exp(ref_log)
            normal = ref > 1e-300
            assert np.all(np.abs(G[i][sample][normal] - ref[normal]) <= eps * ref[normal]), (bi, h)
            inside = ref >= TINY
            btol = bruteforce_tolerance(q64, r64, h)
            assert np.all(np.abs(Gb[i][sample][inside] - ref[inside]) <= btol[inside]), (bi, h)
            checked += len(sample)
            underflow += int((ref_log < np.log(TINY)).sum())
        assert np.all(np.isfinite(L)) and np.all(np.isfinite(G))
    assert checked > 0
    assert underflow > 0  # the sample reaches sums below the float32 range
