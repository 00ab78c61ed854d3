"""Pins of the FP64 network oracle: the convolution against SciPy's
correlation, every backward map against its adjoint identity, and the full
gradient against central finite differences."""

import numpy as np
import pytest
from scipy import signal

from oracle import net_oracle as net


def test_conv3_is_scipy_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((5, 6, 7, 3))
    w = rng.standard_normal((27, 2, 3))
    y = net.conv3(x, w)
    for o in range(2):
        ref = np.zeros(x.shape[:3])
        for c in range(3):
            K = w[:, o, c].reshape(3, 3, 3)            # [dz, dy, dx]
            ref += signal.correlate(x[..., c], K, mode="same")
        np.testing.assert_allclose(y[..., o], ref, rtol=1e-12, atol=1e-12)


def test_conv3_backward_is_adjoint():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((4, 5, 6, 3))
    w = rng.standard_normal((27, 4, 3))
    g = rng.standard_normal((4, 5, 6, 4))
    gx, gw = net.conv3_bwd(x, w, g)
    assert np.isclose(np.sum(net.conv3(x, w) * g), np.sum(x * gx))
    dw = rng.standard_normal(w.shape)
    assert np.isclose(np.sum(net.conv3(x, dw) * g), np.sum(dw * gw))


@pytest.mark.parametrize("shape", [(4, 6, 8, 2), (5, 7, 3, 2)])
def test_pool_and_up_backward_are_adjoint(shape):
    rng = np.random.default_rng(2)
    a = rng.standard_normal(shape)
    pa = net.pool(a)
    b = rng.standard_normal(pa.shape)
    assert np.isclose(np.sum(pa * b), np.sum(a * net.pool_bwd(b, shape)))
    ua = net.up(b, shape)
    g = rng.standard_normal(shape)
    assert np.isclose(np.sum(ua * g), np.sum(b * net.up_bwd(g, b.shape)))


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    Z, Y, X = 6, 5, 7
    mask = (rng.random((Z, Y, X)) > 0.2).astype(float)
    rs = [rng.standard_normal((Z, Y, X)) for _ in range(2)]
    ts = [rng.standard_normal((Z, Y, X)) for _ in range(2)]
    masks = [mask, mask]
    theta = net.init_params(4)
    L, g = net.loss_and_grad(theta, rs, masks, ts)
    assert np.isclose(L, net.loss(theta, rs, masks, ts))
    h = 1e-6
    idx = np.concatenate([rng.integers(0, len(theta), 24), len(theta) - 1 - np.arange(4)])
    for i in idx:
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        fd = (net.loss(tp, rs, masks, ts) - net.loss(tm, rs, masks, ts)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])
    d = rng.standard_normal(len(theta))
    fd = (net.loss(theta + h * d, rs, masks, ts) - net.loss(theta - h * d, rs, masks, ts)) / (2 * h)
    assert np.isclose(fd, g @ d, rtol=1e-5)


def test_strided_pool_matches_pool_and_block_means():
    rng = np.random.default_rng(5)
    a = rng.standard_normal((6, 7, 9))
    np.testing.assert_allclose(net.pool_s(a, 2), net.pool(a[..., None])[..., 0], rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(net.pool_s(a, 4), net.pool_s(net.pool_s(a, 2), 2), rtol=1e-14, atol=1e-14)
    b = rng.standard_normal((8, 8, 12))
    assert np.isclose(net.pool_s(b, 4)[1, 0, 2], b[4:8, 0:4, 8:12].mean())
    assert np.array_equal(net.pool_s(b, 1), b)


@pytest.mark.parametrize("s", [1, 2, 4])
def test_prolong_reproduces_constants_and_linear_functions(s):
    shape = (9, 13, 17)
    C = [-(-n // s) for n in shape]
    yc = np.full(C, 3.25)
    np.testing.assert_allclose(net.prolong(yc, shape, s), 3.25, rtol=1e-15)
    # a linear function of the cell-centre coordinates is reproduced wherever
    # the fine centre lies between two coarse centres
    zc, ycc, xc = np.meshgrid(*[(np.arange(c) + 0.5) * s for c in C], indexing="ij")
    lin = 0.3 * xc - 1.1 * ycc + 0.7 * zc
    out = net.prolong(lin, shape, s)
    zf, yf, xf = np.meshgrid(*[np.arange(n) + 0.5 for n in shape], indexing="ij")
    ref = 0.3 * xf - 1.1 * yf + 0.7 * zf
    inner = tuple(slice(s // 2 + 1, (c - 1) * s + s // 2 - 1 if s > 1 else n) for c, n in zip(C, shape))
    np.testing.assert_allclose(out[inner], ref[inner], rtol=1e-12, atol=1e-12)
    if s == 1:
        np.testing.assert_allclose(out, ref, rtol=1e-14, atol=1e-14)
