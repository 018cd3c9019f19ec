"""Cross-validation scores (the introduction's CV_LK and CV_LS) from the
dual-tree sums against the oracle's exact scores: the difference must lie
within the bound the call returns, which follows from the per-query
guarantee of the sums."""
import numpy as np
import pytest

import oracle
import paper_1102_2878_gb300 as dfgt
from conftest import to_cuda
from paper_1102_2878_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("eps", [1e-2, 1e-3])
def test_cv_scores_within_their_bounds(dev, orc, eps):
    x, _, _ = datagen.workload("kde2d_n1e4")
    hs = [0.005, 0.02, 0.05, 0.2]
    t = dfgt.Tree(dev, to_cuda(x))
    out = dfgt.cv_scores(dev, t, hs, eps)
    x64 = x.astype(np.float64)
    for k, h in enumerate(hs):
        lk, ls = oracle.cv_lk(x64, h), oracle.cv_ls(x64, h)
        # the leave-one-out sums carry |S~ - S| <= eps S, so the CV_LK bound
        # is -log(1 - eps) at every bandwidth, isolated points included,
        # unless some S lies below the float32 range (no neighbour within
        # ~13 h: outside the guarantee, S~ = 0 and the score is -inf)
        S = orc.loo_sums(x64, h)
        if S.min() > 1e-30:
            assert out["lk_bound"][k] == pytest.approx(-np.log1p(-eps), rel=1e-12), (h, out["lk_bound"][k])
            assert abs(out["cv_lk"][k] - lk) <= out["lk_bound"][k] + 1e-12 * abs(lk), (h, out["cv_lk"][k], lk)
        else:
            assert not np.isfinite(out["lk_bound"][k])
        assert abs(out["cv_ls"][k] - ls) <= out["ls_bound"][k] + 1e-12 * abs(ls), (h, out["cv_ls"][k], ls)


def test_cv_scores_agree_with_brute_force_sums(dev):
    # the same scores from the exact GPU sums (S = G - 1), tighter tolerance
    x, _, _ = datagen.workload("kde2d_n1e4")
    hs = [0.01, 0.1]
    t = dfgt.Tree(dev, to_cuda(x))
    out = dfgt.cv_scores(dev, t, hs, 1e-3)
    n, D = x.shape
    for k, h in enumerate(hs):
        G = dfgt.kde_sum_bruteforce(dev, to_cuda(x), to_cuda(x), [h, np.sqrt(2) * h]).cpu().numpy()
        V = (2 * np.pi * h * h) ** (D / 2)
        Vs = (2 * np.pi * 2 * h * h) ** (D / 2)
        lk = np.mean(np.log((G[0] - 1) / ((n - 1) * V)))
        ls = np.mean((G[1] - 1) / ((n - 1) * Vs) - 2 * (G[0] - 1) / ((n - 1) * V))
        assert abs(out["cv_lk"][k] - lk) <= out["lk_bound"][k] + 1e-5
        assert abs(out["cv_ls"][k] - ls) <= out["ls_bound"][k] + 1e-5 * abs(ls)


# ------------------------------------------------------ leave-one-out sums
@pytest.mark.parametrize("D,n,leaf", [(2, 6000, 0), (3, 5000, 32), (1, 3000, 16), (8, 1500, 32)])
@pytest.mark.parametrize("eps", [1e-2, 1e-4])
def test_sum_loo_within_eps_of_the_leave_one_out_sums(dev, orc, D, n, leaf, eps):
    # relative to S itself, so isolated points (S far below 1) are held to eps too
    x = datagen.isotropic_mixture(n, D, 6, 0.05, seed=70 + D).astype(np.float32)
    hs = [0.003, 0.02, 0.1, 0.5]
    t = dfgt.Tree(dev, to_cuda(x), leaf_size=leaf, eps_fp=min(2e-5, eps / 4))
    S, st = dfgt.kde_sum_loo(dev, t, hs, eps)
    S = S.cpu().numpy()
    x64 = x.astype(np.float64)
    for k, h in enumerate(hs):
        want = orc.loo_sums(x64, h)
        ok = want > 1e-30
        err = np.abs(S[k] - want)
        assert np.all(err[ok] <= eps * want[ok]), (h, float((err[ok] / want[ok]).max()))
        assert np.all(np.abs(S[k][~ok]) <= 1e-29)


def test_sum_loo_counts_duplicates_and_not_the_point_itself(dev, orc):
    # every point twice: S_i holds its twin's term 1 and nothing for itself
    base = datagen.isotropic_mixture(700, 2, 3, 0.05, seed=3).astype(np.float32)
    x = np.concatenate([base, base])
    t = dfgt.Tree(dev, to_cuda(x), leaf_size=16)
    for h in (1e-4, 0.03):
        S, _ = dfgt.kde_sum_loo(dev, t, [h], 1e-3)
        S = S.cpu().numpy()[0]
        want = orc.loo_sums(x.astype(np.float64), h)
        assert np.all(np.abs(S - want) <= 1e-3 * want)
        if h == 1e-4:
            assert np.all(S >= 1.0)


def test_sum_loo_rejects_a_single_point(dev):
    t = dfgt.Tree(dev, to_cuda(np.float32([[0.5, 0.5]])))
    with pytest.raises(dfgt.DFGTError):
        dfgt.kde_sum_loo(dev, t, [0.1], 1e-2)
