"""Each summary operator of the GPU path against the oracle, element by element.

dfgt_apply_pairs runs the production action kernels on a chosen list of
node pairs, then the downward local-to-local pass and the leaf read-out.
The oracle evaluates the same truncated expansions by their formulas in
FP64 (far-field moments + evaluation, direct local moments, far-to-local
translation, the distance-bound prune value, the exact leaf sum).  Local
expansions are evaluated by the oracle directly at the query node's center;
the GPU shifts them to the leaves first, which is exact (Lemma 3.6), so the
two agree to rounding.

Tolerance: the GPU evaluates series terms in float32.  With u = 2^-24 the
rounding error of an order-p series is at most c u sum|terms| with
c = 2 (2 p^D + 6 p D + 6 D + 16) (the same allowance the traversal adds to
its truncation bounds); sum|terms| is computed here from the oracle's own
series, so the check is |gpu - oracle| <= c u sum|terms| + 1e-12.  A local
expansion is shifted to the leaf center c' before it is read out, so its
terms are taken at |x - c'| + |c' - c| per dimension (the absolute values
of the shifted polynomial's terms), which is never less than |x - c|.
"""
import math

import numpy as np
import pytest

import paper_1102_2878_gb300 as dfgt
from conftest import to_cuda
from paper_1102_2878_gb300 import _lib, datagen

pytestmark = pytest.mark.gpu
U = 2.0 ** -24


def allowance(p, D):
    return 2 * (2 * p ** D + 6 * p * D + 6 * D + 16) * U


@pytest.fixture(scope="module", params=[1, 2, 3, 4, 5])
def setup(request, dev):
    D = request.param
    x = datagen.isotropic_mixture(4000, D, 5, 0.08, seed=200 + D)
    y = datagen.isotropic_mixture(3000, D, 5, 0.08, seed=300 + D)
    qt = dfgt.Tree(dev, to_cuda(x), leaf_size=24)
    rt = dfgt.Tree(dev, to_cuda(y), leaf_size=24)
    return D, x.astype(np.float64), y.astype(np.float64), qt, rt, qt.export(), rt.export()


def node_points(X, t, j):
    idx = t["perm"][t["begin"][j]:t["begin"][j] + t["count"][j]]
    return idx, X[idx]


def center(t, j):
    return 0.5 * (t["lo"][j].astype(np.float64) + t["hi"][j].astype(np.float64))


def side(t, j):
    return float((t["hi"][j].astype(np.float64) - t["lo"][j].astype(np.float64)).max())


def leaf_centers(t, n):
    """center of the leaf holding each point, in the caller's point order"""
    out = np.zeros((n, t["lo"].shape[1]))
    for j in np.where(t["left"] < 0)[0]:
        out[t["perm"][t["begin"][j]:t["begin"][j] + t["count"][j]]] = center(t, j)
    return out


def pick_nodes(t, rng, k, min_count=40):
    cand = np.where(t["count"] >= min_count)[0]
    return rng.choice(cand, size=min(k, len(cand)), replace=False)


def multi(pm, D):
    """multi-indices of the radix-pm layout, last dimension least significant"""
    idx = np.arange(pm ** D)
    return np.stack([(idx // pm ** (D - 1 - k)) % pm for k in range(D)], axis=1)


def hermite_table(orc, t, n):
    return np.array([orc.hermite_functions(tk, n) for tk in t])  # [D][n]


def series(orc, kind, Rp, Qp, cR, cQ, h, p, pm, cL=None):
    """Oracle value of the truncated series at each query, and the sum of
    the absolute values of its terms (the scale of float32 rounding); cL
    holds the center of each query's leaf, where local expansions are read
    out."""
    D = Rp.shape[1]
    s = 1.0 / np.sqrt(2 * h * h)
    A = multi(pm, D)
    keep = (A < p).all(1)
    fact = np.array([np.prod([math.factorial(int(v)) for v in a]) for a in A])
    # absolute moments sum_r |(r-c)s|^alpha / alpha!
    absM = np.array([(np.abs((Rp - cR) * s) ** a).prod(1).sum() for a in A]) / fact * keep
    if kind == "F":
        want = orc.eval_farfield(orc.farfield_moments(Rp, cR, h, p, pm), cR, h, p, Qp, pm)
        scale = np.zeros(len(Qp))
        for i, q in enumerate(Qp):
            H = np.abs(hermite_table(orc, (q - cR) * s, pm))
            scale[i] = sum(absM[j] * np.prod([H[k, A[j, k]] for k in range(D)]) for j in range(len(A)) if keep[j])
        return want, scale
    if kind == "D":
        L = orc.direct_local(Rp, cQ, h, p, pm)
        absL = np.zeros(len(A))
        for r in Rp:
            H = np.abs(hermite_table(orc, (cQ - r) * s, pm))
            absL += np.array([np.prod([H[k, a[k]] for k in range(D)]) for a in A]) / fact * keep
    else:
        L = orc.far_to_local(orc.farfield_moments(Rp, cR, h, p, pm), cR, cQ, h, p, pm)
        H = np.abs(hermite_table(orc, (cQ - cR) * s, 2 * pm - 1))
        absL = np.zeros(len(A))
        for b in range(len(A)):
            if keep[b]:
                absL[b] = sum(absM[j] * np.prod([H[k, A[j, k] + A[b, k]] for k in range(D)])
                              for j in range(len(A)) if keep[j]) / fact[b]
    want = orc.eval_local(L, cQ, h, p, Qp, pm)
    X = np.abs((Qp - cQ) * s) if cL is None else np.abs((Qp - cL) * s) + np.abs((cL - cQ) * s)
    scale = np.array([(absL * (x[None, :] ** A).prod(1)).sum() for x in X])
    return want, scale


@pytest.mark.parametrize("kind", ["F", "D", "T"])
def test_expansion_operator(setup, orc, dev, kind):
    D, X, Y, qt, rt, tq, tr = setup
    rng = np.random.default_rng(D * 7 + len(kind))
    pm = tq["info"]["p_max"]
    act = {"F": _lib.ACT_FARFIELD, "D": _lib.ACT_LOCAL, "T": _lib.ACT_F2L}[kind]
    for trial in range(3):
        qn = int(pick_nodes(tq, rng, 1)[0])
        rn = int(pick_nodes(tr, rng, 1)[0])
        h = 1.1 * max(side(tq, qn), side(tr, rn))  # keeps every series small (r < 1/2)
        p = int(rng.integers(1, pm + 1))
        G = dfgt.apply_pairs(dev, qt, rt, [qn], [rn], [act], [p], h).cpu().numpy()
        qidx, Qp = node_points(X, tq, qn)
        _, Rp = node_points(Y, tr, rn)
        want, scale = series(orc, kind, Rp, Qp, center(tr, rn), center(tq, qn), h, p, pm,
                             leaf_centers(tq, len(X))[qidx])
        err = np.abs(G[qidx] - want)
        assert np.all(err <= allowance(p, D) * scale + 1e-12), (kind, D, p, err.max(), scale.max())
        others = np.setdiff1d(np.arange(len(X)), qidx)
        assert np.all(G[others] == 0.0)


def test_prune_and_base_operators(setup, orc, dev):
    D, X, Y, qt, rt, tq, tr = setup
    rng = np.random.default_rng(D)
    h = 0.07
    # prune on arbitrary pairs: |R| (K(d^l) + K(d^u)) / 2 for every query of Q
    qn = int(pick_nodes(tq, rng, 1)[0])
    rn = int(pick_nodes(tr, rng, 1)[0])
    G = dfgt.apply_pairs(dev, qt, rt, [qn], [rn], [_lib.ACT_PRUNE], [1], h).cpu().numpy()
    dl, du = orc.dist_bounds(tq["lo"][qn].astype(np.float64), tq["hi"][qn].astype(np.float64),
                             tr["lo"][rn].astype(np.float64), tr["hi"][rn].astype(np.float64))
    val = 0.5 * tr["count"][rn] * (np.exp(-dl * dl / (2 * h * h)) + np.exp(-du * du / (2 * h * h)))
    qidx, _ = node_points(X, tq, qn)
    # the GPU brackets K(d^l), K(d^u) in float32: directed rounding of the
    # exponent x = d^2/2h^2 costs about 3u x relative, expf 2 ulps, plus a
    # 1e-6 margin on each bound
    x = max(dl * dl, du * du) / (2 * h * h)
    assert np.allclose(G[qidx], val, rtol=3e-6 + 4 * U * x, atol=1e-40)
    # base case on leaf pairs: exact sums
    lq = np.where(tq["left"] < 0)[0]
    lr = np.where(tr["left"] < 0)[0]
    qs, rs = rng.choice(lq, 6, replace=False), rng.choice(lr, 6, replace=False)
    G = dfgt.apply_pairs(dev, qt, rt, qs, rs, [_lib.ACT_BASE] * 6, [1] * 6, h).cpu().numpy()
    want = np.zeros(len(X))
    tol = np.zeros(len(X))
    for a, b in zip(qs, rs):
        qi, Qp = node_points(X, tq, a)
        _, Rp = node_points(Y, tr, b)
        want[qi] += orc.naive_kde(Qp, Rp, h)
        # float32 rounding: each term exp(-x) with x = d^2/2h^2 carries the
        # ex2 error (< 2^-21 relative) and either (D+4)u x (direct form) or
        # at most 5e-6 + (4D+8)u x (expanded form, used only when its bound
        # allows); the run of at most 24 terms is summed in float32
        x = ((Qp[:, None, :] - Rp[None, :, :]) ** 2).sum(2) / (2 * h * h)
        K = np.exp(-x)
        tol[qi] += (K * (2.0 ** -21 + (4 * D + 8) * U * x + 5e-6)).sum(1) + 24 * U * K.sum(1)
        # terms below the float32 normal range flush to zero
        tol[qi] += np.where(K < 2.0 ** -125, K, 0.0).sum(1)
    bad = np.abs(G - want) > tol + 1e-300
    assert not bad.any(), (np.flatnonzero(bad)[:5], G[bad][:5], want[bad][:5], tol[bad][:5])
    assert (want > 0).sum() > 0


def test_mixed_list_accumulates(setup, orc, dev):
    """Several kinds on overlapping query nodes: contributions add up."""
    D, X, Y, qt, rt, tq, tr = setup
    rng = np.random.default_rng(99 + D)
    pm = tq["info"]["p_max"]
    qn = pick_nodes(tq, rng, 3, min_count=60)
    rn = pick_nodes(tr, rng, 3, min_count=40)
    h = 1.1 * max(max(side(tq, j) for j in qn), max(side(tr, j) for j in rn))
    acts = [_lib.ACT_FARFIELD, _lib.ACT_LOCAL, _lib.ACT_F2L]
    ps = [pm, max(1, pm - 1), pm]
    G = dfgt.apply_pairs(dev, qt, rt, qn, rn, acts, ps, h).cpu().numpy()
    want = np.zeros(len(X))
    scale = np.zeros(len(X))
    for a, b, act, p in zip(qn, rn, acts, ps):
        qi, Qp = node_points(X, tq, a)
        _, Rp = node_points(Y, tr, b)
        kind = {_lib.ACT_FARFIELD: "F", _lib.ACT_LOCAL: "D", _lib.ACT_F2L: "T"}[act]
        v, sc = series(orc, kind, Rp, Qp, center(tr, b), center(tq, a), h, p, pm,
                       leaf_centers(tq, len(X))[qi])
        want[qi] += v
        scale[qi] += sc
    assert np.all(np.abs(G - want) <= allowance(pm, D) * scale + 1e-12)
