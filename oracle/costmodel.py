"""Float64 CPU oracle of the learned cost model's network -- TEST INFRASTRUCTURE ONLY.

Only tests may import this module; it shares no code with the CUDA kernels. The network
is y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3 with 8 inputs and two hidden layers of 32
units; the loss is L = (1/n) sum_i (y_i - t_i)^2. The parameters are one flat vector in
the library's layout: W1[32][8], b1[32], W2[32][32] (row j = unit j of the second
layer), b2[32], w3[32], b3.

``grad`` is backpropagation written out with matrix products (the chain rule layer by
layer); ``numeric_grad`` is central differences of ``loss``, which shares nothing with it
but the forward pass, and pins it.

Training: ``standardised_labels`` turns item durations (SM cycles) into the regression
targets, log(cycles) shifted by their mean and divided by their population standard
deviation; ``adam_step`` is one update of Adam as Kingma and Ba publish it (ICLR 2015,
Algorithm 1: exponential moving averages of the gradient and of its square, both divided
by one minus their decay raised to the step number, then a step of lr times their
quotient); ``fit`` is that many full-batch Adam steps from given parameters.
"""

from __future__ import annotations

import numpy as np

KF, KH = 8, 32
SIZES = (("W1", KH * KF), ("b1", KH), ("W2", KH * KH), ("b2", KH), ("w3", KH), ("b3", 1))
N_PARAMS = sum(n for _, n in SIZES)


def unpack(p: np.ndarray) -> dict:
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, n in SIZES:
        out[name] = p[o:o + n]
        o += n
    out["W1"] = out["W1"].reshape(KH, KF)
    out["W2"] = out["W2"].reshape(KH, KH)
    out["b3"] = float(out["b3"][0])
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.ravel(np.asarray(d[name], dtype=np.float64)) for name, _ in SIZES])


def forward(p, X):
    """Returns (y, cache) for inputs X [n, 8]."""
    w = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ w["W1"].T + w["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ w["W2"].T + w["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w["w3"] + w["b3"]
    return y, (X, z1, h1, z2, h2, w)


def loss(p, X, t) -> float:
    y, _ = forward(p, X)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def grad(p, X, t):
    """(L, dL/dp) by backpropagation."""
    y, (X, z1, h1, z2, h2, w) = forward(p, X)
    t = np.asarray(t, dtype=np.float64)
    n = X.shape[0]
    r = y - t
    dy = 2.0 * r / n                         # dL/dy_i
    g = {"b3": dy.sum(), "w3": h2.T @ dy}
    dz2 = np.outer(dy, w["w3"]) * (z2 > 0)   # dL/dz2
    g["b2"] = dz2.sum(axis=0)
    g["W2"] = dz2.T @ h1
    dz1 = (dz2 @ w["W2"]) * (z1 > 0)         # dL/dz1
    g["b1"] = dz1.sum(axis=0)
    g["W1"] = dz1.T @ X
    return float(np.mean(r * r)), pack(g)


def numeric_grad(p, X, t, eps: float = 1e-6) -> np.ndarray:
    """Central differences of the loss, one parameter at a time (slow; small n)."""
    p = np.asarray(p, dtype=np.float64).copy()
    out = np.empty_like(p)
    for i in range(p.shape[0]):
        old = p[i]
        p[i] = old + eps
        lp = loss(p, X, t)
        p[i] = old - eps
        lm = loss(p, X, t)
        p[i] = old
        out[i] = (lp - lm) / (2 * eps)
    return out


def standardised_labels(cycles):
    """t_i = (log c_i - mean) / sd over the samples, c_i < 1 read as 1, sd the population
    standard deviation (floored at 1e-6 so that equal durations do not divide by zero).
    Returns (t, mean, sd)."""
    c = np.maximum(np.asarray(cycles, dtype=np.float64), 1.0)
    lg = np.log(c)
    mu = float(lg.mean())
    sd = float(np.sqrt(max(float(np.mean((lg - mu) ** 2)), 1e-12)))
    return (lg - mu) / sd, mu, sd


def adam_step(p, g, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update at step number ``step`` (1 for the first). Returns new (p, m, v)."""
    p = np.asarray(p, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** step)
    v_hat = v / (1.0 - beta2 ** step)
    return p - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def fit(p0, X, cycles, steps: int, lr: float):
    """``steps`` full-batch Adam steps on the mean squared error against the standardised
    log-cycle labels, from parameters p0 and zero moments. Returns (p, final loss, labels)."""
    t, _, _ = standardised_labels(cycles)
    p = np.asarray(p0, dtype=np.float64).copy()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for k in range(1, steps + 1):
        _, g = grad(p, X, t)
        p, m, v = adam_step(p, g, m, v, k, lr)
    return p, loss(p, X, t), t
