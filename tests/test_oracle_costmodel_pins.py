"""Pins of the cost-model oracle (float64 backpropagation): central differences, a
closed form, and a planted mistake. CPU only."""

from __future__ import annotations

import numpy as np
import pytest

from oracle import costmodel as cm


def _case(seed, n=12):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.3, cm.N_PARAMS)
    X = rng.uniform(0, 1.5, (n, cm.KF))
    t = rng.normal(0, 1, n)
    return p, X, t


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_backprop_equals_central_differences(seed):
    p, X, t = _case(seed)
    L, g = cm.grad(p, X, t)
    assert L == pytest.approx(cm.loss(p, X, t), rel=1e-12)
    num = cm.numeric_grad(p, X, t)
    assert np.max(np.abs(g - num)) <= 1e-6 * max(1.0, np.max(np.abs(num)))


def test_constant_network_closed_form():
    """All weights and biases zero but b3 = c: y = c, L = mean((c - t)^2), dL/db3 =
    2 (c - mean t), every other derivative 0 (the ReLUs see 0)."""
    rng = np.random.default_rng(3)
    X = rng.uniform(0, 1, (20, cm.KF))
    t = rng.normal(0, 1, 20)
    p = np.zeros(cm.N_PARAMS)
    p[-1] = 0.7
    L, g = cm.grad(p, X, t)
    assert L == pytest.approx(np.mean((0.7 - t) ** 2), rel=1e-12)
    assert g[-1] == pytest.approx(2 * (0.7 - t.mean()), rel=1e-12)
    assert np.all(g[:-1] == 0)


def test_layout_round_trip():
    p, _, _ = _case(4)
    assert np.array_equal(cm.pack(cm.unpack(p)), p)
    assert cm.N_PARAMS == 1377


def test_a_dropped_relu_mask_fails_the_difference_pin():
    """The pin is sensitive: backprop without the layer-1 ReLU mask disagrees."""
    p, X, t = _case(5)
    y, (Xc, z1, h1, z2, h2, w) = cm.forward(p, X)
    dy = 2.0 * (y - t) / X.shape[0]
    dz2 = np.outer(dy, w["w3"]) * (z2 > 0)
    wrong = (dz2 @ w["W2"]).T @ Xc                # missing (z1 > 0)
    num = cm.numeric_grad(p, X, t)[: cm.KH * cm.KF].reshape(cm.KH, cm.KF)
    assert np.max(np.abs(wrong - num)) > 1e-3


# ------------------------------------------------------------------ training step (Adam)

def test_adam_first_step_moves_by_lr_times_the_sign():
    """From zero moments the bias-corrected averages are g and g^2, so the first step is
    exactly lr * g / (|g| + eps): lr times the sign of g for |g| >> eps, zero for g = 0."""
    g = np.array([3.0, -0.5, 1e-3, 0.0, -7e2])
    p0 = np.array([0.1, 0.2, -0.3, 0.4, 0.5])
    p1, m, v = cm.adam_step(p0, g, np.zeros(5), np.zeros(5), 1, lr=0.01)
    assert np.allclose(p1, p0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_adam_bias_correction_with_a_constant_gradient():
    """With the same gradient every step, m_k = (1 - b1^k) g and v_k = (1 - b2^k) g^2, so
    the corrected averages stay g and g^2 and every step has the same size. Without the
    correction the steps would grow from 0.1 / sqrt(0.001) ~ 3.16 times too large."""
    g = np.array([0.25, -4.0, 2e-2])
    p = np.zeros(3)
    m = np.zeros(3)
    v = np.zeros(3)
    for k in range(1, 51):
        p, m, v = cm.adam_step(p, g, m, v, k, lr=1e-3)
        assert np.allclose(p, -k * 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-9, atol=1e-15)


def test_adam_two_steps_worked_by_hand():
    """g1 = 1 then g2 = -2, lr = 1, beta = (0.9, 0.999), eps = 1e-8, from p = 0:
    step 1: m = 0.1, v = 0.001, corrected 1 and 1, p = -1 / (1 + 1e-8);
    step 2: m = 0.9 * 0.1 - 0.2 = -0.11, v = 0.999 * 0.001 + 0.001 * 4 = 0.004999,
    corrected m = -0.11 / 0.19, v = 0.004999 / 0.001999, and
    p = p1 + (0.11 / 0.19) / (sqrt(0.004999 / 0.001999) + 1e-8)."""
    p, m, v = cm.adam_step([0.0], [1.0], [0.0], [0.0], 1, lr=1.0)
    assert p[0] == pytest.approx(-1.0 / (1.0 + 1e-8), abs=1e-15)
    p, m, v = cm.adam_step(p, [-2.0], m, v, 2, lr=1.0)
    assert m[0] == pytest.approx(-0.11, abs=1e-15)
    assert v[0] == pytest.approx(0.004999, abs=1e-15)
    want = -1.0 / (1.0 + 1e-8) + (0.11 / 0.19) / (np.sqrt(0.004999 / 0.001999) + 1e-8)
    assert p[0] == pytest.approx(want, abs=1e-14)
    assert p[0] == pytest.approx(-1.0 + 0.5789473684 / 1.5813761018, abs=1e-8)


def test_standardised_labels():
    """cycles 1 and 100: logs 0 and ln 100, mean ln 10, sd ln 10, labels -1 and 1;
    durations below one cycle count as one; the labels have mean 0 and variance 1 and do
    not change when every duration is scaled by the same factor."""
    t, mu, sd = cm.standardised_labels([1, 100])
    assert np.allclose(t, [-1.0, 1.0]) and mu == pytest.approx(np.log(10)) and sd == pytest.approx(np.log(10))
    t0, _, _ = cm.standardised_labels([0, -5, 100])
    t1, _, _ = cm.standardised_labels([1, 1, 100])
    assert np.array_equal(t0, t1)
    rng = np.random.default_rng(8)
    c = rng.integers(50, 10**7, 200)
    t, _, _ = cm.standardised_labels(c)
    assert abs(t.mean()) < 1e-12 and np.mean(t * t) == pytest.approx(1.0, rel=1e-12)
    t2, _, _ = cm.standardised_labels(c * 64)
    assert np.allclose(t, t2, rtol=0, atol=1e-12)
    t3, _, sd3 = cm.standardised_labels([77, 77, 77])
    assert np.all(t3 == 0) and sd3 == pytest.approx(1e-6)


def test_fit_lowers_the_loss_and_equals_its_own_steps():
    """fit is labels + full-batch Adam: the same as taking the steps by hand, and on a
    learnable target its loss falls."""
    rng = np.random.default_rng(9)
    X = rng.uniform(0, 1, (64, cm.KF))
    cycles = np.exp(3.0 + 2.0 * X[:, 0] - X[:, 3] + 0.05 * rng.normal(size=64))
    p0 = rng.normal(0, 0.3, cm.N_PARAMS)
    p, L, t = cm.fit(p0, X, cycles, steps=30, lr=3e-3)
    q, m, v = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    for k in range(1, 31):
        _, g = cm.grad(q, X, t)
        q, m, v = cm.adam_step(q, g, m, v, k, 3e-3)
    assert np.array_equal(p, q)
    assert L < 0.8 * cm.loss(p0, X, t)


def test_adam_without_bias_correction_fails_the_constant_gradient_pin():
    """A planted mistake: dropping the correction makes the first step 3.16 lr, not lr."""
    g = np.array([0.5])
    m = 0.1 * g
    v = 0.001 * g * g
    wrong = 0.0 - 1e-3 * m / (np.sqrt(v) + 1e-8)
    right, _, _ = cm.adam_step([0.0], g, [0.0], [0.0], 1, lr=1e-3)
    assert abs(wrong[0] - right[0]) > 1e-3
