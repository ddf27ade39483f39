"""Pins of the oracle's update deltas: brute force before and after, closed forms on
K_{a,b}, round trips, and switching invariance. CPU only."""

from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from tests import _golden


def _random_graph(rng, n_u, n_v, density, p_pos):
    edges = [(a, b, 1 if rng.random() < p_pos else -1)
             for a in range(n_u) for b in range(n_v) if rng.random() < density]
    return _golden.graph(n_u, n_v, edges)


def _random_batch(rng, g, k):
    present = {(a, b): s for a, b, s in zip(g.u.tolist(), g.v.tolist(), g.sign.tolist())}
    cells = [(a, b) for a in range(g.n_u) for b in range(g.n_v)]
    pick = rng.choice(len(cells), size=min(k, len(cells)), replace=False)
    u, v, s = [], [], []
    for i in pick:
        a, b = cells[i]
        if (a, b) in present:
            s.append(int(rng.choice([0, 1, -1])))
        else:
            s.append(int(rng.choice([1, -1])))
        u.append(a)
        v.append(b)
    return np.array(u, np.int32), np.array(v, np.int32), np.array(s, np.int8)


def test_delta_equals_brute_force_before_and_after():
    rng = np.random.default_rng(0)
    for _ in range(40):
        g = _random_graph(rng, 7, 8, 0.55, 0.6)
        u, v, s = _random_batch(rng, g, int(rng.integers(1, 9)))
        h = oracle.apply_updates(g, u, v, s)
        b0, b1 = oracle.brute_force(g), oracle.brute_force(h)
        assert oracle.count_delta(g, u, v, s) == (b1.balanced - b0.balanced, b1.unbalanced - b0.unbalanced)


@pytest.mark.parametrize("a,b", [(3, 4), (5, 5), (6, 3)])
def test_closed_forms_on_complete_bipartite(a, b):
    """Deleting one edge of an all-positive K_{a,b} removes the (a-1)(b-1) butterflies
    through it; flipping it makes them all unbalanced."""
    g = _golden.graph(a, b, [(i, j, 1) for i in range(a) for j in range(b)])
    lost = (a - 1) * (b - 1)
    assert oracle.count_delta(g, [0], [0], [0]) == (-lost, 0)
    assert oracle.count_delta(g, [0], [0], [-1]) == (-lost, lost)
    assert oracle.count_delta(g, [0], [0], [1]) == (0, 0)
    assert math.comb(a, 2) * math.comb(b, 2) - lost == oracle.count(
        oracle.apply_updates(g, [0], [0], [0])).balanced


def test_round_trip_and_switching():
    rng = np.random.default_rng(1)
    for _ in range(10):
        g = _random_graph(rng, 9, 9, 0.5, 0.7)
        u, v, s = _random_batch(rng, g, 6)
        h = oracle.apply_updates(g, u, v, s)
        # undo: restore every touched edge to its old state
        old = {(a, b): x for a, b, x in zip(g.u.tolist(), g.v.tolist(), g.sign.tolist())}
        us = [old.get((a, b), 0) for a, b in zip(u.tolist(), v.tolist())]
        d1 = oracle.count_delta(g, u, v, s)
        d2 = oracle.count_delta(h, u, v, np.array(us, np.int8))
        assert (d1[0] + d2[0], d1[1] + d2[1]) == (0, 0)
        # negating every edge at one vertex (switching) changes nothing
        x = int(rng.integers(0, g.n_u))
        sel = g.u == x
        if sel.any():
            assert oracle.count_delta(g, g.u[sel], g.v[sel], -g.sign[sel]) == (0, 0)


def test_bad_batches_are_rejected():
    g = _golden.graph(2, 2, [(0, 0, 1)])
    with pytest.raises(ValueError):
        oracle.apply_updates(g, [1], [1], [0])           # absent edge
    with pytest.raises(ValueError):
        oracle.apply_updates(g, [0, 0], [1, 1], [1, -1])  # repeated pair
