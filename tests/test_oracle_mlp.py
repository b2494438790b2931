"""Pins of the oracle's h-predictor network (not in the paper): backprop
against central finite differences, forward values of hand-set weights,
the closed form of Adam's first step, and bfloat16 rounding of known values."""
import math

import numpy as np
import pytest


def _theta(orc, seed=0, scale=0.3):
    return np.random.default_rng(seed).normal(scale=scale, size=orc.HNET_NPARAM)


def test_parameter_count(orc):
    assert orc.HNET_NPARAM == 64 * 5 + 64 + 64 * 64 + 64 + 64 + 1


def test_backprop_matches_finite_differences(orc):
    rng = np.random.default_rng(1)
    th = _theta(orc)
    X = rng.normal(size=(16, 5))
    t = rng.normal(size=16)
    _, g = orc.hnet_loss_grad(th, X, t)
    idx = rng.choice(th.size, 200, replace=False)
    for i in idx:
        e = 1e-6
        tp, tm = th.copy(), th.copy()
        tp[i] += e
        tm[i] -= e
        fd = (orc.hnet_loss_grad(tp, X, t)[0] - orc.hnet_loss_grad(tm, X, t)[0]) / (2 * e)
        assert abs(fd - g[i]) < 1e-7 * max(1.0, abs(g[i]))


def test_forward_hand_set_weights(orc):
    th = np.zeros(orc.HNET_NPARAM)
    W1, b1, W2, b2, W3, b3 = orc.hnet_unpack(th)    # views into th
    b3[0] = 0.25
    X = np.array([[1.0, 0.0, 0.0, 0.0, 0.0], [-2.0, 0.0, 0.0, 0.0, 0.0]])
    y, _ = orc.hnet_forward(th, X)
    assert np.all(y == 0.25)
    W1[0, 0] = 1.0
    W2[0, 0] = 1.0
    W3[0, 0] = 1.0
    y, _ = orc.hnet_forward(th, X)

    def silu(v):
        return v / (1.0 + math.exp(-v))
    assert silu(1.0) == pytest.approx(0.7310585786300049, rel=1e-15)
    assert y[0] == pytest.approx(silu(silu(1.0)) + 0.25, rel=1e-14)
    assert y[1] == pytest.approx(silu(silu(-2.0)) + 0.25, rel=1e-14)


def test_prediction_is_gain_times_output(orc):
    th = _theta(orc, 3)
    X = np.random.default_rng(9).normal(size=(7, 5))
    X[2, 3] = 0.0                                   # at rest: no change of h
    y, _ = orc.hnet_forward(th, X)
    s = orc.hnet_predict(th, X)
    assert s[2] == 0.0
    assert np.allclose(s, X[:, 3] * y, rtol=0, atol=0)
    loss, _ = orc.hnet_loss_grad(th, X, np.zeros(7))
    assert loss == pytest.approx(np.mean(s * s), rel=1e-15)


def test_adam_first_step_closed_form(orc):
    rng = np.random.default_rng(4)
    th = rng.normal(size=50)
    g = rng.normal(size=50)
    lr = 1e-3
    th1, m, v = orc.adam_update(th, g, np.zeros(50), np.zeros(50), 1, lr)
    assert np.allclose(th1, th - lr * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_bf16_rounding(orc):
    vals = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -7, -3.0, 1 + 2 ** -8 + 2 ** -20])
    ref = np.array([1.0, 1.0, 1 + 2 ** -6, 1 + 2 ** -7, -3.0, 1 + 2 ** -7])
    assert np.array_equal(orc.bf16_round(vals), ref)
