"""Pins of the proposal-network oracle: its convolution is a library
correlation, its gradient matches central finite differences of the exact
(unrounded) forward, bf16 rounding is round-to-nearest-even, and its Adam step
matches a hand-computed step."""
import numpy as np
import pytest

from oracle import net


def test_conv_is_a_library_correlation():
    rng = np.random.default_rng(1)
    x = rng.normal(size=256)
    theta = net.init_params(3).astype(np.float64)
    z, cc = net.forward(theta, x, rounding=False)
    q = net.unpack(theta)
    for c in range(16):
        ref = np.correlate(np.pad(x, 4), q["W1"][c, 0], mode="valid") + q["b1"][c]
        assert np.allclose(cc["h1"][c], ref, atol=1e-12)
    assert np.isclose(z, q["b4"][0] + q["W4"] @ np.max(np.maximum(cc["h3"], 0), axis=1))


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.normal(size=256) * 2.0
    theta = net.init_params(5).astype(np.float64)
    theta[net.N_PARAMS - 17:net.N_PARAMS - 1] = rng.normal(size=16)  # nonzero head weights
    loss, g = net.backward(theta, x, 1.0, rounding=False)
    idx = rng.choice(net.N_PARAMS, 60, replace=False)
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        lp = net.loss_of(net.forward(tp, x, False)[0], 1.0)
        lm = net.loss_of(net.forward(tm, x, False)[0], 1.0)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * max(1.0, abs(fd)), (i, fd, g[i])


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.0e38, 0.0], np.float32)
    r = net.bf16(v)
    assert r[0] == 1.0 and r[1] == 1.0  # halfway rounds to even (1.0)
    assert r[2] == 1.0 + 2 ** -7        # above halfway rounds up
    assert r[3] == -2.5 and r[5] == 0.0
    assert np.all(np.abs(r - v) <= np.abs(v) * 2 ** -8)


def test_adam_step_by_hand():
    th, m, v = np.array([1.0, -2.0]), np.zeros(2), np.zeros(2)
    g = np.array([0.5, -0.25])
    th1, m1, v1 = net.adam(th, m, v, g, 1, 0.1)
    # first step: m_hat = g, v_hat = g^2, update = lr * sign(g) (up to eps)
    assert np.allclose(th1, th - 0.1 * np.sign(g), atol=1e-7)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)


def test_decimate_closed_forms():
    # a constant row c: every output is (16 c - 16 mu) / (4 sigma) = 4 (c - mu) / sigma
    x = np.full((2, 16 * 7 + 5), 2.5)
    d = net.decimate(x, np.array([0.5, 2.5]), np.array([2.0, 1.0]))
    assert d.shape == (2, 7)
    assert np.allclose(d[0], 4.0 * (2.5 - 0.5) / 2.0) and np.allclose(d[1], 0.0)
    # a ramp x[i] = i: block j sums 16 * 16 j + 120 (the trailing 5 samples are dropped)
    r = np.arange(16 * 7 + 5, dtype=np.float64)[None, :]
    d = net.decimate(r, 0.0, 1.0)
    assert np.allclose(d[0], (256.0 * np.arange(7) + 120.0) / 4.0)


def test_decimate_whitens_gaussian_noise():
    # white noise N(mu, sigma^2) becomes unit-variance, zero-mean blocks; the
    # neighbouring blocks are independent (disjoint sums)
    rng = np.random.default_rng(7)
    mu, sigma = 3.0, 0.7
    x = mu + sigma * rng.normal(size=(1, 16 * 20000))
    d = net.decimate(x, mu, sigma)[0]
    assert abs(d.mean()) < 0.03 and abs(d.var() - 1.0) < 0.03
    assert abs(np.corrcoef(d[:-1], d[1:])[0, 1]) < 0.03
