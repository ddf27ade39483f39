"""GPU parity at the full sizes of the named workloads, in bench.py's launch configuration
(default tuning, per-vertex counts on).

Single graphs: the totals and SHA-256 digests of the per-vertex arrays must equal those the
CPU oracle wrote into tests/golden/full_*.txt (tests/golden/make_full_size.py), and a
sample of per-vertex counts is recomputed one vertex at a time by the oracle. The batched
workload (4,096 graphs): every member against the oracle-written totals of
tests/golden/batch_4096_chung_lu.txt (tests/golden/make_batch_golden.py). The serving mix: a
stream with the full-size large request, every ticket against those goldens.
"""

from __future__ import annotations

import hashlib
import os

import numpy as np
import pytest

import oracle
from paper_2601_17707_gb300 import bbc, synth
from tests import _golden
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


@pytest.mark.parametrize("name", ["powerlaw_1m_200k_20m", "hubs_50k_2m_100m", "serve_large_200k_100k_5m"])
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


def batch_digest(gs):
    h = hashlib.sha256()
    for g in gs:
        h.update(np.ascontiguousarray(g.u, dtype="<i4").tobytes())
        h.update(np.ascontiguousarray(g.v, dtype="<i4").tobytes())
        h.update(np.ascontiguousarray(g.sign, dtype="i1").tobytes())
    return h.hexdigest()


@pytest.fixture(scope="module")
def full_batch():
    head, rows = _golden.load_batch()
    gs = synth.batch_graphs(synth.batch_specs(int(head["graphs"]), seed=int(head["seed"])))
    assert batch_digest(gs) == head["edges_sha256"], "generator drifted from the golden batch"
    return gs, rows


def test_full_size_batch_every_member(gpu_lib, full_batch):
    """All 4,096 members of one bbc_count_batch call (autotuned, as bench.py runs it)
    against the oracle-written totals, member by member, then again on replay."""
    gs, rows = full_batch
    want = [r[3] for r in rows]
    G = [bbc.Graph.from_synthetic(g) for g in gs]
    try:
        bbc.autotune_batch(G)
        got = bbc.count_batch(G)
        bad = [i for i in range(len(gs)) if got[i] != want[i]]
        assert not bad, bad[:10]
        assert bbc.count_batch(G) == want      # replay of the captured plan
        t = bbc.default_tuning()
        assert bbc.count_batch(G, tuning=t) == want
    finally:
        for h in G:
            h.free()


def test_full_size_serving_mix(gpu_lib, full_batch):
    """A stream of batch members with the serving workload's full-size large request
    (|U| = 200,000, |V| = 100,000, 5M edges) submitted twice mid-stream, on the 8 GB budget:
    every ticket equals the oracle-written total of its graph."""
    gs, rows = full_batch
    large_want = _golden.load_full("serve_large_200k_100k_5m")
    large = synth.large_serving_graph(seed=int(large_want["seed"]))
    assert edge_digest(large) == large_want["edges_sha256"]
    idx = list(range(0, len(gs), 13))
    stream = [("b", i) for i in idx]
    stream.insert(20, ("L", -1))
    stream.insert(len(stream) // 2, ("L", -1))
    srv = bbc.Server(8 << 30)
    try:
        tickets = [srv.submit(large if kind == "L" else gs[i]) for kind, i in stream]
        got = [srv.wait(t, timeout_s=300.0) for t in tickets]
        want = [int(large_want["balanced"]) if kind == "L" else rows[i][3] for kind, i in stream]
        bad = [k for k in range(len(stream)) if got[k] != want[k]]
        assert not bad, [stream[k] for k in bad[:10]]
        c = srv.counters()
        assert c["completed"] == len(stream) and c["peak_reserved_bytes"] <= c["budget_bytes"]
    finally:
        srv.close()
