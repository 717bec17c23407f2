"""Pins of the FP64 reference network (oracle/cnn.py) on the CPU."""
import math

import numpy as np
import pytest

from oracle import cnn


def test_conv_matches_scipy_correlate():
    """conv3x3 = zero-padded cross-correlation (library special case)."""
    sp = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(0)
    a = rng.standard_normal((2, 3, 9, 9))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    z = cnn.conv3x3(a, W, b)
    for bi in range(2):
        for co in range(4):
            want = b[co] + sum(sp.correlate2d(a[bi, ci], W[co, ci], mode="same") for ci in range(3))
            np.testing.assert_allclose(z[bi, co], want, rtol=1e-12, atol=1e-12)


def test_gelu_closed_form_and_derivative():
    x = np.linspace(-5, 5, 101)
    np.testing.assert_allclose(cnn.gelu(x), x * 0.5 * (1 + np.vectorize(math.erf)(x / math.sqrt(2))), rtol=1e-13)
    h = 1e-6
    np.testing.assert_allclose(cnn.gelu_grad(x), (cnn.gelu(x + h) - cnn.gelu(x - h)) / (2 * h), rtol=1e-7, atol=1e-9)


def test_gradients_finite_differences():
    """Every parameter gradient of the loss against central differences (small network)."""
    rng = np.random.default_rng(1)
    P, B = 8, 2
    params = cnn.init_params(channels=4, layers=3, seed=2)
    x = rng.standard_normal((B, P, P))
    t = (0.9 + 0.1 * rng.random((B, P, P))) * np.exp(1j * rng.uniform(0, 1.5, (B, P, P)))
    w = rng.random((P, P))
    loss, grads = cnn.loss_and_grads(params, x, t, w)
    h = 1e-6
    for l, (W, b) in enumerate(params):
        for arr, g in ((W, grads[l][0]), (b, grads[l][1])):
            flat = arr.reshape(-1)
            for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + h
                lp, _ = cnn.loss_and_grads(params, x, t, w)
                flat[idx] = old - h
                lm, _ = cnn.loss_and_grads(params, x, t, w)
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - g.reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_head_bounds_and_adam_decreases_loss():
    rng = np.random.default_rng(3)
    P, B = 8, 4
    params = cnn.init_params(channels=4, layers=3, seed=4)
    x = rng.standard_normal((B, P, P))
    o, _ = cnn.forward(params, x)
    assert np.all(np.abs(o) >= 0.8 - 1e-12) and np.all(np.abs(o) <= 1.0 + 1e-12)
    assert np.all(np.angle(o) >= -1e-12) and np.all(np.angle(o) <= math.pi / 2 + 1e-12)
    t = 0.95 * np.exp(0.6j) * np.ones((B, P, P))
    w = np.ones((P, P))
    state = {}
    l0, g = cnn.loss_and_grads(params, x, t, w)
    for _ in range(30):
        params = cnn.adam_step(params, g, state, lr=1e-2)
        l1, g = cnn.loss_and_grads(params, x, t, w)
    assert l1 < 0.5 * l0


def test_stitch_constant_patches():
    """Stitching identical constant patches returns that constant where covered, 1 elsewhere."""
    probe = np.exp(-np.linspace(-2, 2, 8)[:, None] ** 2 - np.linspace(-2, 2, 8)[None] ** 2).astype(complex)
    pos = np.array([[0, 0], [4, 4], [8, 2]])
    c = 0.9 * np.exp(0.3j)
    out = cnn.stitch(np.full((3, 8, 8), c), probe, pos, (20, 20), floor=0.0)
    assert np.allclose(out[:8, :8], c) and out[19, 19] == 1.0


def test_adam_first_step_is_signed_learning_rate():
    """With bias correction the first Adam step moves every parameter by lr * g / (|g| + eps)."""
    rng = np.random.default_rng(5)
    params = cnn.init_params(channels=3, layers=2, seed=6)
    grads = [(rng.standard_normal(W.shape), rng.standard_normal(b.shape)) for W, b in params]
    out = cnn.adam_step(params, grads, {}, lr=0.01, eps=0.0)
    for (W, b), (W1, b1), (gW, gb) in zip(params, out, grads):
        np.testing.assert_allclose(W1 - W, -0.01 * np.sign(gW), rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(b1 - b, -0.01 * np.sign(gb), rtol=1e-12, atol=1e-15)


def test_adam_first_step_with_eps():
    """Kingma & Ba, Algorithm 1: after the bias correction the first step is
    -lr g / (|g| + eps), eps outside the square root; gradients near eps show its place."""
    params = [(np.array([[[[1.0]]]]), np.array([0.0]))]
    grads = [(np.array([[[[3e-8]]]]), np.array([-1e-8]))]
    out = cnn.adam_step(params, grads, {}, lr=0.1, eps=1e-8)
    np.testing.assert_allclose(out[0][0].ravel(), [1.0 - 0.1 * 0.75], rtol=1e-12)
    np.testing.assert_allclose(out[0][1], [0.1 * 0.5], rtol=1e-12)


def test_adam_constant_gradient_second_step():
    """A constant gradient g keeps m_hat = g and v_hat = g^2 at every step, so every step is -lr sign(g)."""
    params = [(np.array([[[[1.0]]]]), np.array([2.0]))]
    grads = [(np.array([[[[0.3]]]]), np.array([-4.0]))]
    state = {}
    p = params
    for _ in range(3):
        p = cnn.adam_step(p, grads, state, lr=0.1, eps=0.0)
    np.testing.assert_allclose(p[0][0].ravel(), [0.7], rtol=1e-12)
    np.testing.assert_allclose(p[0][1], [2.3], rtol=1e-12)


def test_zero_network_predicts_centre_of_ranges():
    """All weights and biases zero: sigmoid(0) = 1/2 gives amplitude 0.9 and phase pi/4 at every
    pixel, so the loss against target 0 is 0.81 and against that value 0."""
    P, B = 6, 3
    params = [(np.zeros_like(W), np.zeros_like(b)) for W, b in cnn.init_params(channels=4, layers=3)]
    x = np.random.default_rng(7).standard_normal((B, P, P))
    o, _ = cnn.forward(params, x)
    np.testing.assert_allclose(o, 0.9 * np.exp(1j * math.pi / 4), rtol=1e-15)
    w = np.random.default_rng(8).random((P, P))
    assert abs(cnn.loss_and_grads(params, x, np.zeros((B, P, P)), w)[0] - 0.81) < 1e-14
    assert cnn.loss_and_grads(params, x, o, w)[0] < 1e-30


def test_features_centre_zero_frequency():
    d = np.zeros((1, 8, 8))
    d[0, 0, 0] = 9.0
    x = cnn.features(d)
    assert x[0, 4, 4] == pytest.approx(math.log(4.0)) and np.count_nonzero(x) == 1
