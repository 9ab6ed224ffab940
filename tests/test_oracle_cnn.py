"""Pins of the CNN oracle: convolution against scipy's 2-D correlation,
gradients against central finite differences, Adam's first step, and the
zero-initialised last layer returning f exactly."""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import cnn


def test_conv_matches_scipy_correlation():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 7, 9, 3))
    w = rng.normal(size=(9, 3, 4))
    b = rng.normal(size=4)
    y = cnn.conv(x, w, b)
    for n in range(2):
        for o in range(4):
            ref = np.full((7, 9), b[o])
            for i in range(3):
                k = w[:, i, o].reshape(3, 3)   # tap = (dy+1)*3 + (dx+1)
                ref += correlate2d(x[n, :, :, i], k, mode="same", boundary="fill", fillvalue=0)
            np.testing.assert_allclose(y[n, :, :, o], ref, rtol=1e-12, atol=1e-12)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    f = rng.random((2, 6, 5))
    ustar = f + 0.1 * rng.normal(size=f.shape)
    theta = cnn.init_params(3, zero_last=False)
    theta += 0.01 * rng.normal(size=theta.size)   # non-zero biases too
    L, g = cnn.gradients(theta, f, ustar)
    assert L == pytest.approx(cnn.loss(theta, f, ustar), rel=1e-14)
    idx = rng.choice(theta.size, size=60, replace=False)
    # make sure every layer is probed
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in cnn.SHAPES])
    idx = np.unique(np.concatenate([idx, offs[:-1], offs[1:] - 1]))
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (cnn.loss(tp, f, ustar) - cnn.loss(tm, f, ustar)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9), i


def test_zero_last_layer_returns_f():
    rng = np.random.default_rng(2)
    f = rng.random((1, 8, 8))
    u0, _ = cnn.forward(cnn.init_params(5), f)
    assert np.array_equal(u0, f)


def test_adam_first_step_moves_by_lr_times_sign():
    """At t = 1 the bias-corrected moments are g and g^2, so every parameter
    moves by lr * g / (|g| + eps), i.e. lr * sign(g) for |g| >> eps."""
    rng = np.random.default_rng(4)
    theta = rng.normal(size=50)
    g = rng.choice([-1.0, 1.0], size=50) * (0.1 + np.abs(rng.normal(size=50)))
    t1, m, v = cnn.adam_step(theta, np.zeros(50), np.zeros(50), g, 1, lr=1e-3)
    np.testing.assert_allclose(theta - t1, 1e-3 * np.sign(g), rtol=1e-6)


def test_parameter_count():
    assert cnn.N_PARAMS == 9 * 32 + 32 + 4 * (9 * 32 * 32 + 32) + 9 * 32 + 1


def test_receptive_field_radius_six():
    """Six 3 x 3 layers with zero padding per layer: the output at a pixel
    depends only on the inputs within Chebyshev radius 6, and the oracle on the
    radius-6 crop (clipped at the image border) gives the same value; one
    input changed at radius 7 leaves it unchanged, at radius 6 changes it."""
    import numpy as np
    from oracle import cnn as ocnn
    rng = np.random.default_rng(4)
    p = ocnn.init_params(3, zero_last=False)
    p[-289:] *= 3.0
    F = rng.random((1, 40, 37))
    u0, _ = ocnn.forward(p, F)
    for r, c in [(0, 0), (20, 18), (39, 36), (5, 30), (0, 20), (39, 0)]:
        r0, c0 = max(0, r - 6), max(0, c - 6)
        crop = F[0, r0:r + 7, c0:c + 7]
        v, _ = ocnn.forward(p, crop[None])
        assert abs(v[0, r - r0, c - c0] - u0[0, r, c]) <= 1e-12
    G = F.copy()
    G[0, 20 + 7, 18] += 1.0
    assert ocnn.forward(p, G)[0][0, 20, 18] == u0[0, 20, 18]
    G = F.copy()
    G[0, 20 + 6, 18 + 6] += 1.0
    assert ocnn.forward(p, G)[0][0, 20, 18] != u0[0, 20, 18]
