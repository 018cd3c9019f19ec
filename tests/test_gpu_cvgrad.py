"""Gradient of CV_LK (dfgt_cv_grad and its autograd wrapper) against the
oracle's float64 gradient and central differences of the exact score."""
import math

import numpy as np
import pytest

import paper_1102_2878_gb300 as dfgt
from conftest import to_cuda
from paper_1102_2878_gb300 import datagen

pytestmark = pytest.mark.gpu

# Kernel values are float32 (ex2.approx: 2^-21 relative, plus (D+4)u x from
# the rounding of the exponent) and every sum is float64, so the scores
# agree with the float64 oracle to ~1e-6 and the gradients to ~1e-6 of the
# sums of |terms| they are made of; the tolerances leave a factor of 100.


def points(n, D, seed):
    return datagen.isotropic_mixture(n, D, 5, 0.08, seed=seed).astype(np.float32)


@pytest.mark.parametrize("D,n", [(1, 800), (2, 1500), (3, 1200), (8, 600)])
def test_cv_grad_matches_oracle(dev, orc, D, n):
    x = points(n, D, 30 + D)
    hs = np.array([0.03, 0.12]) * math.sqrt(D)
    cv, dlogh, dx = dfgt.cv_grad(dev, to_cuda(x), hs)
    dx = dx.cpu().numpy()
    X = x.astype(np.float64)
    for k, h in enumerate(hs):
        want = orc.cv_lk(X, h)
        g, gx = orc.cv_lk_grad(X, h)
        assert abs(cv[k] - want) <= 1e-4 * (1.0 + abs(want)), (h, cv[k], want)
        assert abs(dlogh[k] - g) <= 1e-4 * (1.0 + abs(g)), (h, dlogh[k], g)
        scale = np.abs(gx).max()
        assert np.abs(dx[k] - gx).max() <= 1e-4 * scale, (h, np.abs(dx[k] - gx).max(), scale)


def test_cv_grad_matches_central_differences_of_the_exact_score(dev, orc):
    # the adjoint against the float64 score itself, not the oracle's gradient
    x = points(400, 2, 77)
    h = 0.05
    cv, dlogh, dx = dfgt.cv_grad(dev, to_cuda(x), [h])
    dx = dx.cpu().numpy()[0]
    X = x.astype(np.float64)
    dl = 1e-5
    fd = (orc.cv_lk(X, h * math.exp(dl)) - orc.cv_lk(X, h * math.exp(-dl))) / (2 * dl)
    assert abs(dlogh[0] - fd) <= 1e-3 * (1.0 + abs(fd))
    scale = np.abs(dx).max()
    for i in (0, 13, 250, 399):
        for d in range(2):
            Xp, Xm = X.copy(), X.copy()
            Xp[i, d] += 1e-6
            Xm[i, d] -= 1e-6
            fd = (orc.cv_lk(Xp, h) - orc.cv_lk(Xm, h)) / 2e-6
            assert abs(dx[i, d] - fd) <= 1e-3 * scale, (i, d, dx[i, d], fd)


def test_cv_grad_translation_and_scaling_identities(dev):
    # sum_k dCV/dx_k = 0 and sum_k x_k . dCV/dx_k + dCV/dlog h = -D hold for
    # the computed gradient up to its float32 kernel values
    x = points(1000, 3, 5)
    cv, dlogh, dx = dfgt.cv_grad(dev, to_cuda(x), [0.05, 0.2])
    dx = dx.cpu().numpy()
    X = x.astype(np.float64)
    for k in range(2):
        scale = np.abs(dx[k]).sum()
        assert np.abs(dx[k].sum(0)).max() <= 1e-5 * scale
        assert float((X * dx[k]).sum()) + dlogh[k] == pytest.approx(-3.0, abs=1e-2)


def test_cv_likelihood_autograd(dev):
    torch = pytest.importorskip("torch")
    x = to_cuda(points(700, 2, 9)).requires_grad_(True)
    lh = torch.tensor(np.log([0.04, 0.1]), dtype=torch.float64, requires_grad=True)
    w = torch.tensor([0.3, -1.2], dtype=torch.float64)
    cv = dfgt.cv_likelihood(dev, x, lh)
    (cv * w).sum().backward()
    cv2, dlogh, dx = dfgt.cv_grad(dev, x.detach(), np.exp(lh.detach().numpy()))
    assert np.allclose(cv.detach().numpy(), cv2)
    assert np.allclose(lh.grad.numpy(), w.numpy() * dlogh)
    want = (0.3 * dx[0] - 1.2 * dx[1]).float()
    assert torch.allclose(x.grad, want, rtol=1e-5, atol=1e-7 * float(want.abs().max()))


def test_cv_grad_two_points_closed_form(dev):
    # N = 2: S = K(d) for both points, CV = log K - log V, dCV/dlog h = d^2/h^2 - D,
    # dCV/dx_0 = -(x_0 - x_1) / h^2
    x = np.float32([[0.1, 0.2], [0.15, 0.26]])
    h = 0.08
    cv, dlogh, dx = dfgt.cv_grad(dev, to_cuda(x), [h])
    dx = dx.cpu().numpy()[0]
    X = x.astype(np.float64)
    d2 = float(((X[0] - X[1]) ** 2).sum())
    assert cv[0] == pytest.approx(-d2 / (2 * h * h) - math.log(2 * math.pi * h * h), abs=1e-6)
    assert dlogh[0] == pytest.approx(d2 / (h * h) - 2, abs=1e-5)
    assert np.allclose(dx[0], -(X[0] - X[1]) / (h * h), rtol=1e-5)
    assert np.allclose(dx[1], (X[0] - X[1]) / (h * h), rtol=1e-5)


def test_cv_grad_rejects_bad_arguments(dev):
    x = to_cuda(points(10, 2, 1))
    with pytest.raises(dfgt.DFGTError):
        dfgt.cv_grad(dev, x[:1], [0.1])
    with pytest.raises(dfgt.DFGTError):
        dfgt.cv_grad(dev, x, [0.0])


def test_boundary_name_dfgt_grad_is_the_same_call(dev):
    import ctypes as C

    import torch

    x = to_cuda(points(700, 3, 41))
    hs = np.array([0.05, 0.2])
    cv, dlogh, dx = dfgt.cv_grad(dev, x, hs)
    cv2, dl2 = np.empty(2), np.empty(2)
    dx2 = torch.empty_like(dx)
    dev.order_after_torch()
    st = dev.lib.dfgt_grad(dev.h, C.c_void_p(x.data_ptr()), 700, 3, hs.ctypes.data_as(C.POINTER(C.c_double)), 2,
                           cv2.ctypes.data_as(C.POINTER(C.c_double)), dl2.ctypes.data_as(C.POINTER(C.c_double)),
                           C.c_void_p(dx2.data_ptr()))
    dev.check(st, "dfgt_grad")
    torch.cuda.synchronize()
    assert np.allclose(cv, cv2, rtol=1e-12, atol=0) and np.allclose(dlogh, dl2, rtol=1e-12, atol=1e-15)
    assert torch.allclose(dx, dx2, rtol=1e-12, atol=1e-15)
