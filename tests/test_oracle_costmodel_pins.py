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
