"""GPU parity at the full sizes of the named workloads, in bench.py's launch configuration
(default tuning, per-vertex counts on).

Single graphs: the totals and SHA-256 digests of the per-vertex arrays must equal those the
CPU oracle wrote into tests/golden/full_*.txt (tests/golden/make_full_size.py), and a
sample of per-vertex counts is recomputed one vertex at a time by the oracle. The batched
workload (4,096 graphs): a sample of members is checked against the oracle one by one.
"""

from __future__ import annotations

import hashlib
import os

import numpy as np
import pytest

import oracle
from paper_2601_17707_gb300 import bbc, synth
from tests._golden import GOLDEN

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, f"full_{name}.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split()
            out[k] = v
    return out


def edge_digest(g):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.u, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(g.v, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(g.sign, dtype="i1").tobytes())
    return h.hexdigest()


def digest(a):
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<u8").tobytes()).hexdigest()


@pytest.mark.parametrize("name", ["powerlaw_1m_200k_20m", "hubs_50k_2m_100m"])
def test_full_size_single_graph(gpu_lib, name):
    want = read_golden(name)
    g = synth.WORKLOADS[name](seed=int(want["seed"]))
    assert edge_digest(g) == want["edges_sha256"], "generator drifted from the golden graph"
    G = bbc.Graph.from_synthetic(g)
    try:
        b, ub, pu, pv = G.count(per_vertex=True)
        assert (b, ub) == (int(want["balanced"]), int(want["unbalanced"]))
        pu, pv = bbc.as_uint64(pu), bbc.as_uint64(pv)
        assert digest(pu) == want["per_u_sha256"]
        assert digest(pv) == want["per_v_sha256"]
        assert int(pu.sum()) == int(want["per_u_sum"]) == 2 * b
        # vertices recomputed one at a time by the oracle (low degree keeps this quick)
        rng = np.random.default_rng(0)
        du = np.bincount(g.u, minlength=g.n_u)
        dv = np.bincount(g.v, minlength=g.n_v)
        for side, deg, arr in ((0, du, pu), (1, dv, pv)):
            cand = np.nonzero((deg >= 2) & (deg <= 40))[0]
            for x in rng.choice(cand, size=min(3, cand.size), replace=False).tolist():
                assert oracle.vertex(g, side, x) == int(arr[x])
    finally:
        G.free()


def test_full_size_batch_sampled(gpu_lib):
    specs = synth.batch_specs(4096, seed=0)
    gs = synth.batch_graphs(specs)
    G = [bbc.Graph.from_synthetic(g) for g in gs]
    try:
        got = bbc.count_batch(G)
        assert len(got) == 4096
        rng = np.random.default_rng(1)
        small = [i for i, g in enumerate(gs) if g.n_edges <= 60_000]
        sample = sorted(rng.choice(small, size=14, replace=False).tolist())
        for i in sample:
            assert got[i] == oracle.count(gs[i], threads=8, per_vertex=False).balanced, i
        assert bbc.count_batch(G) == got      # replay
    finally:
        for h in G:
            h.free()
