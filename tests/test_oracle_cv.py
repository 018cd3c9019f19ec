"""Pins of the oracle's density normalisation and cross-validation scores
(the introduction's Eq. 1, CV_LK and CV_LS) against closed forms,
numerical integration and invariances."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle


@pytest.mark.parametrize("D", [1, 2, 3])
def test_gauss_volume_is_the_integral(D):
    h = 0.37
    f = lambda *z: math.exp(-sum(t * t for t in z) / (2 * h * h))  # noqa: E731
    lim = [(-12 * h, 12 * h)] * D
    val = integrate.nquad(f, lim, opts={"epsabs": 1e-12, "epsrel": 1e-10})[0]
    assert oracle.gauss_volume(D, h) == pytest.approx(val, rel=1e-8)


def test_convolution_kernel_is_sqrt2_h():
    # the normalised convolution of two normalised Gaussians of deviation h
    # is the normalised Gaussian of deviation sqrt(2) h (1-D numerically)
    h = 0.21
    V = oracle.gauss_volume(1, h)
    Vs = oracle.gauss_volume(1, math.sqrt(2) * h)
    for x in (0.0, 0.1, 0.35, 0.8):
        conv = integrate.quad(lambda y: math.exp(-(x - y) ** 2 / (2 * h * h)) * math.exp(-y * y / (2 * h * h)),
                              -3, 3, epsabs=1e-13)[0] / (V * V)
        want = math.exp(-x * x / (2 * 2 * h * h)) / Vs
        assert conv == pytest.approx(want, rel=1e-9)


@pytest.mark.parametrize("D", [1, 2, 3])
def test_two_points_closed_form(D):
    rng = np.random.default_rng(D)
    X = rng.random((2, D))
    h = 0.3
    d2 = float(((X[0] - X[1]) ** 2).sum())
    V = (2 * math.pi * h * h) ** (D / 2)
    Vs = (2 * math.pi * 2 * h * h) ** (D / 2)
    K = math.exp(-d2 / (2 * h * h))
    Ks = math.exp(-d2 / (4 * h * h))
    assert oracle.cv_lk(X, h) == pytest.approx(math.log(K / V), rel=1e-13)
    assert oracle.cv_ls(X, h) == pytest.approx(Ks / Vs - 2 * K / V, rel=1e-12)


def test_three_points_by_hand():
    X = np.array([[0.0], [1.0], [3.0]])
    h = 1.0
    e = lambda d: math.exp(-d * d / 2)  # noqa: E731
    S = [e(1) + e(3), e(1) + e(2), e(3) + e(2)]
    V = math.sqrt(2 * math.pi)
    want = sum(math.log(s / (2 * V)) for s in S) / 3
    assert oracle.cv_lk(X, h) == pytest.approx(want, rel=1e-13)


def test_loo_sums_are_sums_without_self():
    rng = np.random.default_rng(3)
    X = rng.random((40, 3))
    h = 0.2
    assert np.allclose(oracle.loo_sums(X, h), oracle.naive_kde(X, X, h) - 1.0, rtol=1e-13, atol=1e-15)


def test_invariances():
    rng = np.random.default_rng(4)
    X = rng.random((60, 2))
    h, s = 0.15, 2.5
    lk, ls = oracle.cv_lk(X, h), oracle.cv_ls(X, h)
    perm = rng.permutation(len(X))
    assert oracle.cv_lk(X[perm], h) == pytest.approx(lk, rel=1e-13)
    assert oracle.cv_ls(X[perm] + 0.7, h) == pytest.approx(ls, rel=1e-11)
    # densities scale by s^-D when points and bandwidth scale by s
    assert oracle.cv_lk(s * X, s * h) == pytest.approx(lk - 2 * math.log(s), rel=1e-12)
    assert oracle.cv_ls(s * X, s * h) == pytest.approx(ls / s ** 2, rel=1e-11)


# ------------------------------------------------------ gradient of CV_LK
@pytest.mark.parametrize("D,h", [(1, 0.05), (2, 0.08), (3, 0.15)])
def test_cv_lk_grad_log_h_central_difference(D, h):
    rng = np.random.default_rng(10 + D)
    X = rng.random((60, D))
    g, _ = oracle.cv_lk_grad(X, h)
    dl = 1e-4
    fd = (oracle.cv_lk(X, h * math.exp(dl)) - oracle.cv_lk(X, h * math.exp(-dl))) / (2 * dl)
    assert g == pytest.approx(fd, rel=1e-6, abs=1e-8)


@pytest.mark.parametrize("D,h", [(1, 0.05), (2, 0.08), (3, 0.15)])
def test_cv_lk_grad_points_central_difference(D, h):
    rng = np.random.default_rng(20 + D)
    X = rng.random((50, D))
    _, dx = oracle.cv_lk_grad(X, h)
    dl = 1e-6
    for k in (0, 7, 31):
        for d in range(D):
            Xp, Xm = X.copy(), X.copy()
            Xp[k, d] += dl
            Xm[k, d] -= dl
            fd = (oracle.cv_lk(Xp, h) - oracle.cv_lk(Xm, h)) / (2 * dl)
            assert dx[k, d] == pytest.approx(fd, rel=1e-5, abs=1e-7), (k, d)


def test_cv_lk_grad_translation_and_scaling_identities():
    # CV_LK(X + t, h) = CV_LK(X, h): the point gradients sum to zero; and
    # CV_LK(sX, sh) = CV_LK(X, h) - D log s: sum_k x_k . dx_k + dCV/dlog h = -D
    rng = np.random.default_rng(5)
    for D in (1, 2, 4):
        X = rng.normal(size=(45, D))
        g, dx = oracle.cv_lk_grad(X, 0.4)
        scale = np.abs(dx).sum()
        assert np.abs(dx.sum(0)).max() <= 1e-12 * scale
        assert float((X * dx).sum()) + g == pytest.approx(-D, abs=1e-10)
