"""GPU parity of bbc_count_motif: the sign classes of Sec. VII (Table 7) and balanced
(2,k)-bicliques (Def. 5) against the oracle, element by element and exactly, with the pair
side forced either way, both orientations, several counter widths (8/16/32-bit tiles)
and several tiles per anchor.
"""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2601_17707_gb300 import bbc, synth
from tests import _golden

pytestmark = pytest.mark.gpu

SIDES = ((0, bbc.SIDE_FORCE_U), (1, bbc.SIDE_FORCE_V))


def _check(g, kinds=("classes", 2, 3, 4), flags=0, threads=8, sides=SIDES):
    for side, force in sides:
        G = bbc.Graph.from_synthetic(g, flags=flags | force)
        try:
            assert G.info().side == side
            for kind in kinds:
                if kind == "classes":
                    assert G.count_motif("classes") == oracle.motif(g, "classes", side=side,
                                                                    threads=threads)
                else:
                    assert G.count_motif("biclique", k=kind) == \
                        oracle.motif(g, "biclique", k=kind, side=side, threads=threads)
            # the ordinary count still agrees after the motif lists were built
            c = oracle.count(g, threads=threads, per_vertex=False)
            assert G.count()[:2] == (c.balanced, c.unbalanced)
        finally:
            G.free()


def test_fig9_classes_on_the_gpu(gpu_lib):
    g, e = _golden.load("fig9_drug_target.txt")
    G = bbc.Graph.from_synthetic(g, flags=bbc.SIDE_FORCE_U)
    try:
        assert list(G.count_motif("classes")) == e["classes_u"]
    finally:
        G.free()


@pytest.mark.parametrize("seed", [0, 1])
def test_uniform_motifs(gpu_lib, seed):
    _check(synth.uniform_graph(300, 400, 6_000, 0.6, seed=seed))


def test_powerlaw_motifs_several_tiles_and_widths(gpu_lib):
    # hubs of degree > 255 (16-bit counters) and endpoint ranges of several tiles
    _check(synth.powerlaw_1m_200k(seed=3, scale=0.02))


def test_hub_graph_32bit_counters(gpu_lib):
    # a 3 x 70,000 biclique, 90 % positive, pairs on U: each pair shares 70,000 centres,
    # more than 16-bit counters hold -> 32-bit tiles (the V side would visit 7e9 wedges)
    n_u, n_v = 3, 70_000
    u = np.repeat(np.arange(n_u, dtype=np.int32), n_v)
    v = np.tile(np.arange(n_v, dtype=np.int32), n_u)
    rng = np.random.default_rng(1)
    s = np.where(rng.random(u.shape[0]) < 0.9, 1, -1).astype(np.int8)
    g = synth.SignedBipartite(n_u, n_v, u, v, s)
    _check(g, kinds=("classes", 2, 3), threads=8, sides=SIDES[:1])


def test_orientation_and_empty(gpu_lib):
    g = synth.uniform_graph(120, 90, 2_500, 0.5, seed=7)
    _check(g, kinds=("classes", 3), flags=bbc.ORIENT_LOW_ANCHOR)
    empty = synth.SignedBipartite(5, 6, np.zeros(0, np.int32), np.zeros(0, np.int32),
                                  np.zeros(0, np.int8))
    G = bbc.Graph.from_synthetic(empty)
    try:
        assert G.count_motif("classes") == (0,) * 6
        assert G.count_motif("biclique", k=5) == (0, 0)
    finally:
        G.free()


def test_overflow_and_bad_arguments(gpu_lib):
    n_v = 200
    u = np.repeat(np.arange(2, dtype=np.int32), n_v)
    v = np.tile(np.arange(n_v, dtype=np.int32), 2)
    g = synth.SignedBipartite(2, n_v, u, v, np.ones(u.shape[0], np.int8))
    G = bbc.Graph.from_synthetic(g, flags=bbc.SIDE_FORCE_U)
    try:
        with pytest.raises(bbc.BBCError) as e:
            G.count_motif("biclique", k=100)              # C(200, 100) > 2^64
        assert e.value.status == 5
        assert G.count_motif("biclique", k=199) == (200, 200)
        with pytest.raises(bbc.BBCError) as e:
            G.count_motif("biclique", k=1)
        assert e.value.status == 1
    finally:
        G.free()
