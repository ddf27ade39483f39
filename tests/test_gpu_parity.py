"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, bit for bit.

Counts are exact integers, so the tolerance is zero: global balanced / unbalanced totals
and every per-vertex count must equal the oracle's.
"""

from __future__ import annotations

import ctypes

import numpy as np
import pytest

import oracle
from paper_2601_17707_gb300 import bbc, synth
from tests import _golden

pytestmark = pytest.mark.gpu


def gpu_counts(g, flags=0, tuning=None, per_vertex=True, device_input=True):
    G = bbc.Graph.from_synthetic(g, flags=flags, device=device_input)
    try:
        b, ub, pu, pv = G.count(per_vertex=per_vertex, tuning=tuning)
        if per_vertex:
            pu, pv = bbc.as_uint64(pu), bbc.as_uint64(pv)
        return b, ub, pu, pv, G.info()
    finally:
        G.free()


def assert_parity(g, flags=0, tuning=None, want=None, device_input=True):
    want = want or oracle.count(g, threads=4)
    b, ub, pu, pv, info = gpu_counts(g, flags, tuning, device_input=device_input)
    assert (b, ub) == (want.balanced, want.unbalanced)
    np.testing.assert_array_equal(pu, want.per_u)
    np.testing.assert_array_equal(pv, want.per_v)
    return info


def tuning(**kw):
    t = bbc.default_tuning()
    for k, v in kw.items():
        setattr(t, k, v)
    return t


# ------------------------------------------------------------------ paper figures

def test_paper_figures(gpu_lib):
    for name in ("fig1b_signed_k44.txt", "fig9_drug_target.txt"):
        g, e = _golden.load(name)
        b, ub, pu, pv, _ = gpu_counts(g)
        assert (b, ub) == (e["balanced"], e["unbalanced"])
        assert pu.tolist() == e["per_u"] and pv.tolist() == e["per_v"]
    for name, g, label in _golden.load_cases("fig2_butterflies.txt"):
        b, ub, _, _, _ = gpu_counts(g)
        assert (b, ub) == ((1, 0) if label == "balanced" else (0, 1)), name


def test_every_sign_pattern_of_k33(gpu_lib):
    pairs = [(i, j) for i in range(3) for j in range(3)]
    for mask in range(0, 1 << 9, 7):
        edges = [(i, j, -1 if (mask >> k) & 1 else 1) for k, (i, j) in enumerate(pairs)]
        assert_parity(_golden.graph(3, 3, edges))


# ------------------------------------------------------------------ paths and tilings

@pytest.mark.parametrize("seed", range(6))
def test_random_graphs_all_paths(gpu_lib, seed):
    rng = np.random.default_rng(100 + seed)
    n_u = int(rng.integers(30, 400))
    n_v = int(rng.integers(30, 400))
    n_e = int(rng.integers(200, min(n_u * n_v // 3, 20000)))
    dmax_u = min(n_v, max(60, 3 * n_e // n_u))
    dmax_v = min(n_u, max(80, 3 * n_e // n_v))
    g = synth.chung_lu_graph(n_u, n_v, n_e, 2.2, 2.0, dmax_u, dmax_v, float(rng.uniform(0.3, 0.9)),
                             seed=seed)
    want = oracle.count(g)
    # default tuning, dense tiles only, hash only where possible, many tiny tiles and
    # splits, one block per SM, both orientations and both pair sides
    for t in (None, tuning(warp_max_wedges=1), tuning(warp_max_wedges=512),
              tuning(tile_words=1024, split_wedges=64), tuning(blocks_per_sm=1, tile_words=53248),
              tuning(plain=1), tuning(plain=1, tile_words=1024), tuning(group_warps=8),
              tuning(group_warps=8, queue_chunk=7)):
        assert_parity(g, tuning=t, want=want)
    for flags in (bbc.ORIENT_LOW_ANCHOR, bbc.SIDE_FORCE_U, bbc.SIDE_FORCE_V,
                  bbc.SIDE_FORCE_V | bbc.ORIENT_LOW_ANCHOR):
        assert_parity(g, flags=flags, tuning=tuning(tile_words=1024), want=want)


def test_uniform_2k_3k_full_size(gpu_lib):
    g = synth.uniform_2k_3k(seed=0)
    info = assert_parity(g)
    assert info.n_edges == 20000


@pytest.mark.parametrize("scale", [0.003, 0.01])
def test_power_law_shape_scaled(gpu_lib, scale):
    g = synth.powerlaw_1m_200k(seed=1, scale=scale)
    want = oracle.count(g, threads=8)
    assert_parity(g, want=want)
    assert_parity(g, tuning=tuning(tile_words=2048), want=want)
    assert_parity(g, tuning=tuning(plain=1), want=want)
    assert_parity(g, flags=bbc.ORIENT_LOW_ANCHOR, want=want)


def test_heavy_hub_shape_scaled(gpu_lib):
    g = synth.hubs_50k_2m(seed=2, scale=0.005)
    want = oracle.count(g, threads=8)
    assert_parity(g, want=want)
    assert_parity(g, tuning=tuning(tile_words=1024, split_wedges=5000), want=want)


def test_wide_counters_beyond_16_bits(gpu_lib):
    """Anchors sharing more than 65,535 centres take the 32-bit counter tiles."""
    rng = np.random.default_rng(5)
    n_v = 70_000
    edges_u, edges_v = [], []
    for u in range(3):
        edges_u.append(np.full(n_v, u, dtype=np.int32))
        edges_v.append(np.arange(n_v, dtype=np.int32))
    u = np.concatenate(edges_u)
    v = np.concatenate(edges_v)
    s = np.where(rng.random(u.shape[0]) < 0.6, 1, -1).astype(np.int8)
    g = synth.SignedBipartite(3, n_v, u, v, s)
    assert_parity(g)
    assert_parity(g, flags=bbc.ORIENT_LOW_ANCHOR)


# ------------------------------------------------------------------ edge cases

def test_degenerate_graphs(gpu_lib):
    cases = [
        _golden.graph(0, 0, []),
        _golden.graph(7, 3, []),
        _golden.graph(4, 4, [(1, 2, -1)]),
        _golden.graph(1, 300, [(0, j, 1) for j in range(300)]),          # star
        _golden.graph(300, 1, [(i, 0, -1) for i in range(300)]),         # star, other side
        _golden.graph(50, 60, [(i, i, 1) for i in range(50)]),            # matching
        _golden.graph(2, 2, [(0, 0, 1), (0, 1, 1), (1, 0, 1), (1, 1, -1)]),
    ]
    for g in cases:
        assert_parity(g)


def test_host_and_device_inputs_agree(gpu_lib):
    g = synth.powerlaw_1m_200k(seed=4, scale=0.002)
    want = oracle.count(g)
    assert_parity(g, want=want, device_input=False)
    assert_parity(synth.shuffled(g, seed=3), want=want)


def test_invalid_inputs_are_reported(gpu_lib):
    lib = gpu_lib
    def prep(n_u, n_v, edges, flags=0):
        g = _golden.graph(n_u, n_v, edges)
        h = ctypes.c_void_p()
        st = lib.bbc_prepare(n_u, n_v, len(edges), g.u.ctypes.data, g.v.ctypes.data,
                             g.sign.ctypes.data, flags, None, ctypes.byref(h))
        if st == 0:
            lib.bbc_graph_free(h)
        return st
    assert prep(2, 2, [(0, 2, 1)]) == 2          # out of range
    assert prep(2, 2, [(-1, 0, 1)]) == 2
    assert prep(2, 2, [(0, 1, 0)]) == 3          # bad sign
    assert prep(2, 2, [(0, 1, 1), (0, 1, -1)]) == 4   # duplicate
    assert prep(2, 2, [(0, 1, 1), (0, 1, -1)], bbc.DEDUP_LAST) == 0


def test_dedup_keeps_the_last_occurrence(gpu_lib):
    rng = np.random.default_rng(8)
    g = synth.uniform_graph(120, 90, 2500, 0.6, seed=8)
    dup = rng.integers(0, g.n_edges, size=600)
    u = np.concatenate([g.u, g.u[dup]])
    v = np.concatenate([g.v, g.v[dup]])
    s = np.concatenate([-g.sign, g.sign[dup]])  # the earlier copies carry the opposite sign
    order = rng.permutation(u.shape[0])
    # after the permutation, the kept sign of each pair is the one appearing last
    u, v, s = u[order], v[order], s[order]
    key = u.astype(np.int64) * g.n_v + v
    last = {}
    for i, k in enumerate(key.tolist()):
        last[k] = i
    keep = np.array(sorted(last.values()))
    deduped = synth.SignedBipartite(g.n_u, g.n_v, u[keep], v[keep], s[keep])
    want = oracle.count(deduped)
    messy = synth.SignedBipartite(g.n_u, g.n_v, u, v, s)
    info = assert_parity(messy, flags=bbc.DEDUP_LAST, want=want)
    assert info.n_edges == keep.shape[0]


def test_side_choice_follows_wedge_cost(gpu_lib):
    g = synth.powerlaw_1m_200k(seed=0, scale=0.01)
    du = np.bincount(g.u, minlength=g.n_u).astype(np.int64)
    dv = np.bincount(g.v, minlength=g.n_v).astype(np.int64)
    cost_u = int((dv * (dv - 1) // 2).sum())  # pairs on U visit wedges through V
    cost_v = int((du * (du - 1) // 2).sum())
    G = bbc.Graph.from_synthetic(g)
    info = G.info()
    G.free()
    assert info.side == (0 if cost_u <= cost_v else 1)
    assert info.wedges == min(cost_u, cost_v)


def test_work_statistics_cover_every_wedge(gpu_lib):
    """The per-path work behind the bench's per-kernel fractions: over the four paths the
    anchors' oriented wedges add up to W, and their pair-side edges to at most |E|; the
    sum does not depend on the tuning that split the paths."""
    g = synth.powerlaw_1m_200k(seed=9, scale=0.02)
    G = bbc.Graph.from_synthetic(g)
    try:
        W = G.info().wedges
        work = G.work()
        assert sum(w for _, w, _ in work.values()) == W
        assert sum(e for _, _, e in work.values()) <= g.n_edges
        t = bbc.default_tuning()
        t.warp_max_wedges = 1
        t.tile_words = 2048
        G.count(tuning=t)                                   # rebuilds the lists
        assert sum(w for _, w, _ in G.work().values()) == W
    finally:
        G.free()
