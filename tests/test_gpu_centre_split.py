"""GPU parity of centre-split tiles: anchors with more wedges than their tiles can spread
over the blocks have each tile's centres cut into parts whose counts are merged in global
memory. Small split thresholds force the split on small graphs; totals and every
per-vertex count must equal the oracle's, for 8-, 16- and 32-bit counter tiles, one and
several tiles per anchor, repeated counts and batches (and, under the same small split,
the low-anchor orientation, whose light anchors stay whole).
"""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2601_17707_gb300 import bbc, synth

pytestmark = pytest.mark.gpu


def _tuning(**kw):
    t = bbc.default_tuning()
    for k, v in kw.items():
        setattr(t, k, v)
    return t


def _hub_graph(seed=1, hubs=10, d_lo=3_000, d_hi=12_000):
    """20,000 pair-side (U) vertices over 30,000 centres: ten hubs of 3,000 to 12,000
    centres (pairs of hubs share hundreds: 16-bit counters), 200 vertices of 300 centres
    and the rest of 5, so that a hub's endpoint range holds a 16-bit tile and an 8-bit
    one with small tiles."""
    rng = np.random.default_rng(seed)
    n_u, n_v = 20_000, 30_000
    us, vs = [], []
    for x, d in enumerate(np.linspace(d_lo, d_hi, hubs).astype(int)):
        us.append(np.full(d, x))
        vs.append(rng.choice(n_v, size=d, replace=False))
    for x in range(hubs, hubs + 200):
        us.append(np.full(300, x))
        vs.append(rng.choice(n_v, size=300, replace=False))
    rest = np.arange(hubs + 200, n_u)
    us.append(np.repeat(rest, 5))
    vs.append(rng.integers(0, n_v, size=5 * rest.size))
    key = np.unique(np.concatenate(us) * n_v + np.concatenate(vs))
    u = (key // n_v).astype(np.int32)
    v = (key % n_v).astype(np.int32)
    sign = np.where(rng.random(key.size) < 0.6, 1, -1).astype(np.int8)
    return synth.SignedBipartite(n_u, n_v, u, v, sign)


def _wide_graph():
    """60,000 pair-side vertices over 70,000 centres; vertex 0 on every centre and vertex 1
    on 66,000 of them: the two share more than 65,535 centres (32-bit counters)."""
    rng = np.random.default_rng(8)
    n_u, n_v = 60_000, 70_000
    us = [np.zeros(n_v, np.int64), np.ones(66_000, np.int64)]
    vs = [np.arange(n_v), np.arange(66_000)]
    for x in range(2, 102):
        us.append(np.full(300, x))
        vs.append(rng.choice(n_v, size=300, replace=False))
    rest = np.arange(102, n_u)
    us.append(np.repeat(rest, 3))
    vs.append(rng.integers(0, n_v, size=3 * rest.size))
    key = np.unique(np.concatenate(us) * n_v + np.concatenate(vs))
    u = (key // n_v).astype(np.int32)
    v = (key % n_v).astype(np.int32)
    sign = np.where(rng.random(key.size) < 0.6, 1, -1).astype(np.int8)
    return synth.SignedBipartite(n_u, n_v, u, v, sign)


def _split_parts(G):
    """Tile items that share an anchor and a first tile with another item: only parts of
    one centre-split tile do (feature 4 is the item's first tile over the anchor's tiles)."""
    X = G.item_features().cpu().numpy()
    a = G.item_anchors().cpu().numpy()
    keys = list(zip(a.tolist(), np.round(X[:, 4], 6).tolist()))
    seen, dup = set(), 0
    for k in keys:
        dup += k in seen
        seen.add(k)
    return dup


def _check(g, want, flags, tuning, expect_split=True):
    G = bbc.Graph.from_synthetic(g, flags=flags)
    try:
        for _ in range(2):   # the merge buffers are cleared before every count
            b, ub, pu, pv = G.count(per_vertex=True, tuning=tuning)
            assert (b, ub) == (want.balanced, want.unbalanced)
            np.testing.assert_array_equal(bbc.as_uint64(pu), want.per_u)
            np.testing.assert_array_equal(bbc.as_uint64(pv), want.per_v)
            assert G.count(tuning=tuning)[:2] == (want.balanced, want.unbalanced)
        if expect_split:
            assert _split_parts(G) > 0
    finally:
        G.free()


@pytest.mark.parametrize("tile_words", [0, 4096])
def test_hub_tiles_split_by_centres(gpu_lib, tile_words):
    g = _hub_graph()
    want = oracle.count(g, threads=8)
    _check(g, want, bbc.SIDE_FORCE_U, _tuning(split_wedges=20_000, tile_words=tile_words))


def test_low_anchor_orientation(gpu_lib):
    g = _hub_graph(seed=2)
    want = oracle.count(g, threads=8)
    _check(g, want, bbc.SIDE_FORCE_U | bbc.ORIENT_LOW_ANCHOR, _tuning(split_wedges=20_000, tile_words=4096),
           expect_split=False)


def test_32_bit_tiles_split_by_centres(gpu_lib):
    g = _wide_graph()
    want = oracle.count(g, threads=8)
    _check(g, want, bbc.SIDE_FORCE_U, _tuning(split_wedges=50_000))


def test_default_split_leaves_small_graphs_alone(gpu_lib):
    g = _hub_graph(seed=3)
    G = bbc.Graph.from_synthetic(g, flags=bbc.SIDE_FORCE_U)
    try:
        G.count()
        assert _split_parts(G) == 0
    finally:
        G.free()


def test_batch_with_split_members(gpu_lib):
    gs = [_hub_graph(seed=4), synth.uniform_graph(300, 200, 5_000, 0.6, seed=5), _hub_graph(seed=6)]
    want = [oracle.count(g, threads=8, per_vertex=False).balanced for g in gs]
    G = [bbc.Graph.from_synthetic(g, flags=bbc.SIDE_FORCE_U) for g in gs]
    try:
        t = _tuning(split_wedges=20_000)
        for _ in range(2):
            assert bbc.count_batch(G, tuning=t) == want
    finally:
        for h in G:
            h.free()


def test_serving_parts_across_ticks(gpu_lib):
    """The serving loop takes a bounded number of a request's tile items per tick, so parts
    of one centre-split tile can run in different launches; the merged counters are cleared
    once per request and the last part, in whichever tick, completes the tile."""
    gs = [_hub_graph(seed=7, hubs=60, d_lo=2_048, d_hi=8_000), _hub_graph(seed=8, hubs=60, d_lo=2_048, d_hi=8_000)]
    want = [oracle.count(g, threads=8, per_vertex=False).balanced for g in gs]
    srv = bbc.Server(4 << 30, tuning=_tuning(split_wedges=20_000, tile_words=4096, blocks_per_sm=1))
    try:
        tickets = [srv.submit(g) for g in gs]
        assert [srv.wait(t, timeout_s=120.0) for t in tickets] == want
        assert max(srv.request_info(t)["ticks"] for t in tickets) >= 2
    finally:
        srv.close()
