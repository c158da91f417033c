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


def test_zero_last_layer_with_the_previous_base_is_the_previous_vector():
    """Base e = 0: an untrained (zero last layer) network reproduces the paper's guess g1, and the
    training target is the step's change in units of s1."""
    rng = np.random.default_rng(4)
    layers = cnn.unpack(pack_random(rng, 0.3))
    layers[-1] = (np.zeros_like(layers[-1][0]), np.zeros_like(layers[-1][1]))
    params = cnn.pack(layers)
    g = [rng.standard_normal((4, 9)) + 1j * rng.standard_normal((4, 9)) for _ in range(4)]
    np.testing.assert_allclose(cnn.guess(params, *g[:3], e=0.0), g[0], atol=1e-14)
    _, tgt, _, s1 = cnn.features(*g[:3], gt=g[3], e=0.0)
    np.testing.assert_allclose(tgt[0] + 1j * tgt[1], (g[3] - g[0]) / np.sqrt(np.mean(np.abs(g[0] - g[1]) ** 2)),
                               rtol=1e-12)


def test_bf16_rounding_is_round_to_nearest_even():
    ulp = 2.0 ** -7                      # BF16 spacing in [1, 2)
    vals = np.array([1.0, 1 + ulp / 2, 1 + 1.5 * ulp, 1 + 0.75 * ulp, -(1 + 0.25 * ulp), 3 + 2 * ulp / 2 + ulp / 4])
    want = np.array([1.0, 1.0, 1 + 2 * ulp, 1 + ulp, -1.0, 3 + 2 * ulp])     # ties to the even neighbour
    np.testing.assert_array_equal(cnn.bf16(vals), want)
    assert abs(cnn.bf16(3.0e38) / 3.0e38 - 1) < 2 ** -8


def test_adam_steps_with_a_constant_gradient():
    """Bias correction makes m_hat = g and v_hat = g^2 for a constant gradient, so every step moves
    each weight by lr g / (|g| + eps)."""
    rng = np.random.default_rng(5)
    w0 = rng.standard_normal(50)
    g = rng.standard_normal(50)
    w, m, v = w0.copy(), np.zeros(50), np.zeros(50)
    for t in range(1, 4):
        w, m, v = cnn.adam_step(w, g, m, v, t, lr=1e-3)
        np.testing.assert_allclose(w, w0 - t * 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_bf16_operands_stay_close_to_fp64():
    rng = np.random.default_rng(6)
    params = pack_random(rng, 0.3)
    x = rng.standard_normal((6, 5, 7))
    tgt = rng.standard_normal((2, 5, 7))
    l64, g64 = cnn.loss_grad(params, x, tgt)
    l16, g16 = cnn.loss_grad(params, x, tgt, bf16_ops=True)
    assert abs(l16 - l64) < 3e-2 * l64
    assert np.linalg.norm(g16 - g64) < 3e-2 * np.linalg.norm(g64)
    # already-BF16 inputs and weights with BF16 rounding switched off reproduce the FP64 path
    out64, _ = cnn.forward(cnn.bf16(params), cnn.bf16(x))
    out16, _ = cnn.forward(cnn.bf16(params), cnn.bf16(x), bf16_ops=True)
    assert np.linalg.norm(out16 - out64) < 2e-2 * np.linalg.norm(out64)
