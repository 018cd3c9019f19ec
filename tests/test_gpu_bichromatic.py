"""Bichromatic D=32 workload: a reference set and uneven query batches
drawn separately from one 128-component mixture, 16 bandwidths, eps 1e-2
and 1e-3 (a smaller case of kde32d_r1e6_q64batches: 1e5 references, six
batches of 1e3..2e4 queries).

Each batch is summed against one reference tree.  The GPU brute force
covers every query and is checked against the FP64 oracle on a seeded
sample; the dual-tree result must be within eps of the oracle wherever the
exact sum is inside the float32 range of the guarantee (G >= 1e-30), and
below it must itself be that small.

Float32 tolerance.  A term exp(-x) computed in float32 from D coordinate
differences carries about (D+3) u x of relative error (u = 2^-24), so at
D = 32, where these sums are made of terms with x of 30..60, the brute
force is checked against sum_r K_r (2^-21 + (D+3) u x_r) + 2^-20 G, and the
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
        tol[i] = (K * (2.0 ** -21 + (D + 3) * U * x)).sum()
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
    checked = 0
    for bi, qx in enumerate(batches[: 6 if eps_index == 0 else 3]):
        qt = dfgt.Tree(dev, to_cuda(qx), eps_fp=EPS_FP)
        G, st = dfgt.kde_sum(dev, qt, rt, hs, eps)
        Gb = dfgt.kde_sum_bruteforce(dev, to_cuda(qx), to_cuda(refs), hs)
        G, Gb = G.cpu().numpy(), Gb.cpu().numpy()
        sample = rng.choice(len(qx), size=12, replace=False)
        q64 = qx.astype(np.float64)[sample]
        for i, h in enumerate(hs):
            ref = orc.naive_kde(q64, r64, h)
            inside = ref >= TINY
            btol = bruteforce_tolerance(q64, r64, h)
            assert np.all(np.abs(Gb[i][sample][inside] - ref[inside]) <= btol[inside]), (bi, h)
            assert np.all(np.abs(G[i][sample][inside] - ref[inside]) <= eps * ref[inside]), (bi, h)
            assert np.all(np.abs(G[i][sample][~inside]) <= 2 * TINY), (bi, h)
            big = Gb[i] >= TINY
            relb = np.abs(G[i][big] - Gb[i][big]) / Gb[i][big]
            # both within their bounds of the exact sum: eps and the brute force's rounding
            assert relb.size == 0 or relb.max() <= eps + EPS_FP, (bi, h, relb.max())
            assert np.all(np.abs(G[i][~big]) <= 2 * TINY), (bi, h)
            checked += int(big.sum())
    assert checked > 0
