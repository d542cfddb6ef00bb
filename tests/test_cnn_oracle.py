"""Pins of the classifier oracle: finite differences, the parameter count the
configuration states (about 20k), and closed forms of the layers."""
import numpy as np
import pytest

from oracle import cnn
from paper_1503_01405_gb300 import synth


def test_parameter_count():
    assert cnn.n_params() == 3 * (32 * 32 * 7 + 32) + 32 * 4 + 4 == 21732


def test_conv_against_direct_sum():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 32, 16))
    w = rng.standard_normal((32, 32, 7))
    b = rng.standard_normal(32)
    y = cnn.conv1d(x, w, b)
    n, co, t = 1, 5, 2
    want = b[co] + sum(w[co, ci, k] * x[n, ci, t + k - 3] for ci in range(32) for k in range(7)
                       if 0 <= t + k - 3 < 16)
    assert abs(y[n, co, t] - want) < 1e-9


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    theta = cnn.init_params(synth.uniform(7, 0, 0, cnn.n_params()))
    theta[32 * 32 * 7: 32 * 32 * 7 + 32] = 0.05        # nonzero biases so ReLUs sit off the kink
    x = rng.standard_normal((3, 32, 32))
    y = np.array([0, 2, 3])
    loss, g, _ = cnn.backward(theta, x, y)
    idx = rng.choice(len(theta), 60, replace=False)
    idx = np.r_[idx, np.arange(len(theta) - 132, len(theta), 11)]
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        lp = cnn.softmax_xent(cnn.forward(tp, x)[0], y)[0]
        lm = cnn.softmax_xent(cnn.forward(tm, x)[0], y)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 + 1e-4 * abs(fd), (i, fd, g[i])


def test_softmax_xent_uniform_logits():
    loss, d, p = cnn.softmax_xent(np.zeros((5, 4)), np.array([0, 1, 2, 3, 0]))
    assert abs(loss - np.log(4)) < 1e-12 and np.allclose(p, 0.25)
    assert np.allclose(d.sum(axis=1), 0)


def test_adam_first_step_moves_by_lr():
    th, m, v = cnn.adam_step(np.zeros(3), np.zeros(3), np.zeros(3), np.array([1.0, -2.0, 0.5]), 1, 0.01)
    assert np.allclose(th, [-0.01, 0.01, -0.01], atol=1e-9)
