"""Pins of the CNN oracle (the learned interface guess): the convolution equals scipy's 2D
cross-correlation, and the analytic gradient equals central finite differences."""
import numpy as np
import pytest

from oracle import cnn


def random_params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return pack_random(rng, scale)


def pack_random(rng, scale):
    layers = [(scale * rng.standard_normal((co, ci, 3, 3)), 0.1 * rng.standard_normal(co)) for ci, co in cnn.LAYERS]
    return cnn.pack(layers)


def test_conv_matches_scipy_correlate2d():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 6, 9))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = cnn.conv3x3(x, w, b)
    for o in range(4):
        ref = b[o] + sum(signal.correlate2d(x[c], w[o, c], mode="same", boundary="fill") for c in range(3))
        np.testing.assert_allclose(y[o], ref, atol=1e-12)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    params = pack_random(rng, 0.3)
    x = rng.standard_normal((6, 5, 7))
    tgt = rng.standard_normal((2, 5, 7))
    loss, g = cnn.loss_grad(params, x, tgt)
    idx = rng.choice(params.size, 40, replace=False)
    eps = 1e-6
    for i in idx:
        pp = params.copy()
        pm = params.copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (cnn.loss_grad(pp, x, tgt)[0] - cnn.loss_grad(pm, x, tgt)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_zero_last_layer_is_linear_extrapolation():
    rng = np.random.default_rng(3)
    params = pack_random(rng, 0.3)
    layers = cnn.unpack(params)
    layers[-1] = (np.zeros_like(layers[-1][0]), np.zeros_like(layers[-1][1]))
    params = cnn.pack(layers)
    g = [rng.standard_normal((4, 9)) + 1j * rng.standard_normal((4, 9)) for _ in range(3)]
    np.testing.assert_allclose(cnn.guess(params, *g), 2 * g[0] - g[1], atol=1e-14)
