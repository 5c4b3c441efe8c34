"""Pins for the closure-network oracle (oracle/closure_net.py), each against
something other than its own formulas: a library correlation, shifts,
textbook normal-CDF values, finite differences and Adam's closed-form first
step."""
import math

import numpy as np
import pytest

from oracle import closure_net as cn
from paper_1807_01769_gb300 import inputs


def _params(seed, scale=1.0, channels=cn.CHANNELS):
    p = inputs.random_phys((cn.num_params(channels),), seed)
    return scale * p


def test_num_params():
    assert cn.num_params() == (32 * 9 + 32) + 2 * (32 * 32 * 9 + 32) + (32 * 9 + 1)


def test_conv_matches_library_periodic_correlation():
    ndimage = pytest.importorskip("scipy.ndimage")
    a = inputs.random_phys((2, 3, 7, 10), 1)
    w = inputs.random_phys((4, 3, 3, 3), 2)
    b = inputs.random_phys((4,), 3)
    got = cn.conv(a, w, b)
    for bi in range(2):
        for co in range(4):
            ref = b[co] + sum(ndimage.correlate(a[bi, ci], w[co, ci], mode="wrap") for ci in range(3))
            np.testing.assert_allclose(got[bi, co], ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("dy,dx", [(-1, -1), (0, 1), (1, 0), (1, -1)])
def test_delta_kernel_is_a_periodic_shift(dy, dx):
    a = inputs.random_phys((1, 1, 5, 6), 4)
    w = np.zeros((1, 1, 3, 3))
    w[0, 0, dy + 1, dx + 1] = 1.0
    got = cn.conv(a, w, None)[0, 0]
    h, wd = a.shape[-2:]
    for y in range(h):
        for x in range(wd):
            assert got[y, x] == a[0, 0, (y + dy) % h, (x + dx) % wd]


def test_gelu_values():
    # Phi(1) = 0.841344746068543, Phi(-1) = 0.158655253931457 (standard normal tables)
    assert abs(cn.gelu(1.0) - 0.841344746068543) < 1e-14
    assert abs(cn.gelu(-1.0) + 0.158655253931457) < 1e-14
    assert cn.gelu(0.0) == 0.0
    z = np.linspace(-6, 6, 49)
    np.testing.assert_allclose(cn.gelu(z) - cn.gelu(-z), z, atol=1e-14)  # Phi(z) + Phi(-z) = 1
    assert abs(cn.gelu(10.0) - 10.0) < 1e-15 and abs(cn.gelu(-10.0)) < 1e-15


def test_gelu_grad_by_finite_differences():
    z = np.linspace(-4, 4, 33)
    h = 1e-6
    fd = (cn.gelu(z + h) - cn.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(cn.gelu_grad(z), fd, atol=1e-8)


def test_forward_is_translation_equivariant():
    p = _params(5, 0.2)
    x = inputs.random_phys((1, 8, 12), 6)
    y, _ = cn.forward(p, x)
    y2, _ = cn.forward(p, np.roll(x, (3, -5), axis=(1, 2)))
    np.testing.assert_allclose(y2, np.roll(y, (3, -5), axis=(1, 2)), atol=1e-12)


def test_gradients_by_finite_differences():
    ch = (1, 3, 4, 2, 1)  # same code path, fewer channels so every parameter is checked
    p = _params(7, 0.4, ch)
    x = inputs.random_phys((2, 5, 6), 8)
    t = inputs.random_phys((2, 5, 6), 9)
    g, l0 = cn.gradients(p, x, t, ch)
    assert abs(l0 - cn.loss(p, x, t, ch)) < 1e-15
    h = 1e-6
    fd = np.empty_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        fd[i] = (cn.loss(p + e, x, t, ch) - cn.loss(p - e, x, t, ch)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)


def test_gradients_full_network_sampled():
    p = _params(10, 0.1)
    x = inputs.random_phys((1, 6, 6), 11)
    t = inputs.random_phys((1, 6, 6), 12)
    g, _ = cn.gradients(p, x, t)
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.choice(p.size, 40, replace=False), [p.size - 1, cn.num_params() - 33]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (cn.loss(p + e, x, t) - cn.loss(p - e, x, t)) / (2 * h)
        assert abs(g[i] - fd) <= 1e-6 * max(1.0, abs(fd)), (i, g[i], fd)


def test_adam_first_step_is_lr_times_sign():
    g = np.array([3.0, -0.5, 1e-3, -7.0])
    p0 = np.zeros(4)
    p1, m, v = cn.adam_step(p0, g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    # m_hat = g, v_hat = g^2 after bias correction, so the step is lr g / (|g| + eps)
    np.testing.assert_allclose(p1, -0.01 * np.sign(g), rtol=1e-5)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_adam_minimises_a_quadratic():
    p = np.array([2.0, -3.0])
    m = v = np.zeros(2)
    for k in range(1, 3001):
        p, m, v = cn.adam_step(p, 2.0 * (p - np.array([0.5, 1.0])), m, v, k, lr=0.01)
    np.testing.assert_allclose(p, [0.5, 1.0], atol=1e-3)
    assert math.isfinite(p.sum())
