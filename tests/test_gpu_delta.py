"""GPU parity of bbc_count_delta (count changes of a batch of edge updates) with the
oracle's before/after counts, exactly: inserts, deletions and sign flips, at hubs and at
random, both pair sides and orientations, host and device inputs, and the errors.
"""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2601_17707_gb300 import bbc, synth

pytestmark = pytest.mark.gpu


def _batch(rng, g, k, hub_bias=False):
    """k distinct updates: flips and deletions of present edges, insertions of absent
    ones; with hub_bias the U endpoints are drawn in proportion to degree squared."""
    present = {(a, b): s for a, b, s in zip(g.u.tolist(), g.v.tolist(), g.sign.tolist())}
    nbrs = {}
    for a, b in present:
        nbrs.setdefault(a, []).append(b)
    deg_u = np.bincount(g.u, minlength=g.n_u).astype(np.float64)
    weight = (deg_u ** 2 if hub_bias else np.ones(g.n_u)) + 1e-12
    p_u = weight / weight.sum()
    out, seen = [], set()
    while len(out) < k:
        a = int(rng.choice(g.n_u, p=p_u))
        if rng.random() < 0.5 and a in nbrs:
            b = int(nbrs[a][int(rng.integers(0, len(nbrs[a])))])     # an existing edge
        else:
            b = int(rng.integers(0, g.n_v))
        if (a, b) in seen:
            continue
        seen.add((a, b))
        if (a, b) in present:
            out.append((a, b, int(rng.choice([0, -present[(a, b)], present[(a, b)]]))))
        else:
            out.append((a, b, int(rng.choice([1, -1]))))
    u, v, s = zip(*out)
    return np.array(u, np.int32), np.array(v, np.int32), np.array(s, np.int8)


def _check(g, u, v, s, flags=0, device=False):
    want = oracle.count_delta(g, u, v, s, threads=8)
    G = bbc.Graph.from_synthetic(g, flags=flags)
    try:
        if device:
            import torch

            got = G.count_delta(torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda(),
                                torch.from_numpy(s).cuda())
        else:
            got = G.count_delta(u, v, s)
        assert got == want
        # the graph is unchanged: a count afterwards is the old count
        c = oracle.count(g, threads=8, per_vertex=False)
        assert G.count()[:2] == (c.balanced, c.unbalanced)
    finally:
        G.free()


@pytest.mark.parametrize("flags", [0, bbc.SIDE_FORCE_U, bbc.SIDE_FORCE_V, bbc.ORIENT_LOW_ANCHOR])
def test_uniform_batches(gpu_lib, flags):
    rng = np.random.default_rng(1)
    g = synth.uniform_graph(150, 120, 3_000, 0.6, seed=3)
    for k in (1, 7, 60):
        _check(g, *_batch(rng, g, k), flags=flags)


def test_powerlaw_batches_at_hubs(gpu_lib):
    rng = np.random.default_rng(2)
    g = synth.powerlaw_1m_200k(seed=4, scale=0.01)
    _check(g, *_batch(rng, g, 40, hub_bias=True))
    _check(g, *_batch(rng, g, 400), device=True)


def _wide_graph():
    """60,000 pair-side (U) vertices over 70,000 centres, so that an anchor's endpoint range
    spans several counter tiles: vertex 0 on every centre and vertex 1 on 66,000 of them
    (counts past 65,535: 32-bit counters), 100 vertices on 300 centres each (16-bit), the
    rest on three centres each (8-bit)."""
    rng = np.random.default_rng(8)
    n_u, n_v = 60_000, 70_000
    us = [np.zeros(n_v, np.int64), np.ones(66_000, np.int64)]
    vs = [np.arange(n_v), np.arange(66_000)]
    mid = rng.choice(np.arange(2, n_u), size=100, replace=False)
    for x in mid:
        us.append(np.full(300, x))
        vs.append(rng.choice(n_v, size=300, replace=False))
    rest = np.setdiff1d(np.arange(2, n_u), mid)
    us.append(np.repeat(rest, 3))
    vs.append(rng.integers(0, n_v, size=3 * rest.size))
    key = np.unique(np.concatenate(us) * n_v + np.concatenate(vs))
    u = (key // n_v).astype(np.int32)
    v = (key % n_v).astype(np.int32)
    sign = np.where(rng.random(key.size) < 0.6, 1, -1).astype(np.int8)
    return synth.SignedBipartite(n_u, n_v, u, v, sign), mid


def test_wide_anchors_over_several_tiles_and_counter_widths(gpu_lib):
    """Updates at the two hubs (32-bit counters), at 300-centre vertices (16-bit) and at
    light ones (8-bit), on a pair side wider than one counter tile."""
    g, mid = _wide_graph()
    rng = np.random.default_rng(9)
    present = {(a, b): s for a, b, s in zip(g.u.tolist(), g.v.tolist(), g.sign.tolist())}
    picks = [(0, 5), (0, 69_999), (1, 10), (1, 67_000)] + [(int(x), int(rng.integers(0, g.n_v))) for x in mid[:20]]
    picks += [(int(a), int(rng.integers(0, g.n_v))) for a in rng.integers(2, g.n_u, size=30)]
    out, seen = [], set()
    for a, b in picks:
        if (a, b) in seen:
            continue
        seen.add((a, b))
        if (a, b) in present:
            out.append((a, b, int(rng.choice([0, -present[(a, b)]]))))
        else:
            out.append((a, b, int(rng.choice([1, -1]))))
    u, v, s = (np.array(x, dt) for x, dt in zip(zip(*out), (np.int32, np.int32, np.int8)))
    _check(g, u, v, s, flags=bbc.SIDE_FORCE_U)


def test_switching_a_vertex_changes_nothing(gpu_lib):
    g = synth.uniform_graph(200, 100, 4_000, 0.5, seed=5)
    x = int(np.bincount(g.u).argmax())
    sel = g.u == x
    G = bbc.Graph.from_synthetic(g)
    try:
        assert G.count_delta(g.u[sel], g.v[sel], (-g.sign[sel]).astype(np.int8)) == (0, 0)
        assert G.count_delta(np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int8)) == (0, 0)
    finally:
        G.free()


def test_bad_batches_are_rejected(gpu_lib):
    g = synth.uniform_graph(50, 40, 600, 0.5, seed=6)
    present = set(zip(g.u.tolist(), g.v.tolist()))
    absent = next((a, b) for a in range(50) for b in range(40) if (a, b) not in present)
    G = bbc.Graph.from_synthetic(g)
    try:
        cases = [
            (([50], [0], [1]), 2),                                 # id out of range
            (([0], [0], [3]), 3),                                  # bad sign
            (([int(g.u[0])] * 2, [int(g.v[0])] * 2, [1, -1]), 4),  # repeated pair
            (([absent[0]], [absent[1]], [0]), 1),                  # deleting an absent edge
        ]
        for (u, v, s), status in cases:
            with pytest.raises(bbc.BBCError) as e:
                G.count_delta(np.array(u, np.int32), np.array(v, np.int32), np.array(s, np.int8))
            assert e.value.status == status
    finally:
        G.free()
