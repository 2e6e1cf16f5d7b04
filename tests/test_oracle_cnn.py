"""Pins for the CPU oracle of the warm-start network: the convolution against a library
correlation, GELU against its limits and a finite difference, the backward pass against
central finite differences of the loss, and the first Adam step in closed form."""
import numpy as np
import pytest
import scipy.signal

from oracle import cnn


def _params(rng, cin=3, ch=4):
    shapes = [(ch, cin, 3, 3), (ch,), (ch, ch, 3, 3), (ch,), (ch, ch, 3, 3), (ch,), (2, ch, 3, 3), (2,)]
    return [0.3 * rng.standard_normal(s) for s in shapes]


def test_conv_matches_library_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 7, 9))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = cnn.conv3x3(x, w, b)
    for bi in range(2):
        for o in range(4):
            ref = b[o] + sum(scipy.signal.correlate2d(x[bi, c], w[o, c], mode="same") for c in range(3))
            assert np.allclose(y[bi, o], ref, atol=1e-12)


def test_dilated_conv_matches_library_correlation_with_spread_kernel():
    rng = np.random.default_rng(5)
    x = rng.standard_normal((1, 2, 13, 11))
    w = rng.standard_normal((3, 2, 3, 3))
    b = np.zeros(3)
    for d in (2, 4):
        y = cnn.conv3x3(x, w, b, d)
        for o in range(3):
            ref = 0.0
            for c in range(2):
                k = np.zeros((2 * d + 1, 2 * d + 1))
                k[::d, ::d] = w[o, c]
                ref = ref + scipy.signal.correlate2d(x[0, c], k, mode="same")
            assert np.allclose(y[0, o], ref, atol=1e-12)


def test_gelu_limits_and_derivative():
    z = np.linspace(-6, 6, 101)
    g = cnn.gelu(z)
    assert abs(cnn.gelu(np.array([0.0]))[0]) == 0.0
    assert np.allclose(g[z > 5], z[z > 5], atol=1e-5) and np.allclose(g[z < -5], 0.0, atol=1e-5)
    h = 1e-6
    assert np.allclose(cnn.gelu_grad(z), (cnn.gelu(z + h) - cnn.gelu(z - h)) / (2 * h), atol=1e-8)


@pytest.mark.parametrize("dil", [(1, 1, 1, 1), (1, 2, 4, 2)])
def test_backward_matches_finite_differences(dil):
    rng = np.random.default_rng(1)
    params = _params(rng)
    net = cnn.CNN(params, dil)
    x = rng.standard_normal((2, 3, 6, 5))
    mask = np.zeros((2, 6, 5))
    mask[0, 1:-1, 1:-1] = 1.0
    mask[1, :-1, :-1] = 1.0
    target = rng.standard_normal((2, 2, 6, 5)) * mask[None]
    loss, grads = net.loss_and_grads(x, mask, target)
    h = 1e-6
    for k in range(8):
        p = net.params[k]
        for _ in range(3):
            idx = tuple(rng.integers(0, s) for s in p.shape)
            old = p[idx]
            p[idx] = old + h
            lp, _ = cnn.CNN(net.params, dil).loss_and_grads(x, mask, target)
            p[idx] = old - h
            lm, _ = cnn.CNN(net.params, dil).loss_and_grads(x, mask, target)
            p[idx] = old
            assert abs((lp - lm) / (2 * h) - grads[k][idx]) <= 1e-6 * max(1.0, abs(grads[k][idx]))


def test_first_adam_step_closed_form():
    # after one step m_hat = g and v_hat = g^2, so w moves by lr * g / (|g| + eps)
    params = [np.array([1.0, -2.0])]
    g = [np.array([0.5, -3.0])]
    m, v = [np.zeros(2)], [np.zeros(2)]
    params, m, v = cnn.adam_step(params, g, m, v, 1, lr=0.1)
    assert np.allclose(params[0], [1.0 - 0.1 * 0.5 / (0.5 + 1e-8), -2.0 + 0.1 * 3.0 / (3.0 + 1e-8)])
