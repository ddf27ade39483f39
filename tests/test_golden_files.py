"""The oracle-written goldens of the full-size workloads, checked on the CPU: the batch
file's member sizes follow the generator's recipe, its sums add up, and a sample of its
members (the smallest ones, so that this stays quick) is recounted by the oracle; the
single-graph files are self-consistent (per-vertex sums equal twice the balanced total,
as every butterfly holds two vertices of each side)."""

from __future__ import annotations

import os

import pytest

import oracle
from paper_2601_17707_gb300 import synth
from tests import _golden


def test_batch_golden_follows_the_recipe_and_recounts():
    head, rows = _golden.load_batch()
    assert int(head["graphs"]) == len(rows) == 4096
    specs = synth.batch_specs(len(rows), seed=int(head["seed"]))
    assert [(s.n_u, s.n_v, s.n_edges) for s in specs] == [r[:3] for r in rows]
    assert sum(r[3] for r in rows) == int(head["balanced_sum"])
    assert sum(r[4] for r in rows) == int(head["unbalanced_sum"])
    small = sorted(range(len(rows)), key=lambda i: rows[i][2])[:6]
    for i in small:
        c = oracle.count(synth.batch_graph(specs[i]), per_vertex=False)
        assert (c.balanced, c.unbalanced) == rows[i][3:], i


@pytest.mark.parametrize("name", ["powerlaw_1m_200k_20m", "hubs_50k_2m_100m", "uniform_2k_3k_20k",
                                  "serve_large_200k_100k_5m"])
def test_full_size_goldens_are_consistent(name):
    want = _golden.load_full(name)
    assert int(want["per_u_sum"]) == int(want["per_v_sum"]) == 2 * int(want["balanced"])
    assert want["workload"] == name


def test_uniform_golden_recounts():
    g = synth.uniform_2k_3k(seed=0)
    want = _golden.load_full("uniform_2k_3k_20k")
    c = oracle.count(g)
    assert (c.balanced, c.unbalanced) == (int(want["balanced"]), int(want["unbalanced"]))
