"""GPU tests of the batched form (bbc_count_batch, bbc_autotune_batch) and the serving
loop (bbc_server_*): every count must equal the oracle's / the single-graph count exactly.
"""

from __future__ import annotations

import ctypes

import numpy as np
import pytest

import oracle
from paper_2601_17707_gb300 import bbc, synth
from tests import _golden

pytestmark = pytest.mark.gpu


def small_batch(n, seed, e_max=20_000):
    specs = synth.batch_specs(n, seed=seed, e_max=e_max)
    return [synth.batch_graph(s) for s in specs]


@pytest.fixture(scope="module")
def batch_graphs():
    gs = small_batch(48, seed=3)
    gs.append(synth.SignedBipartite(10, 12, np.zeros(0, np.int32), np.zeros(0, np.int32),
                                    np.zeros(0, np.int8)))
    gs.append(synth.SignedBipartite(1, 300, np.zeros(300, np.int32), np.arange(300, dtype=np.int32),
                                    np.ones(300, np.int8)))
    gs.append(synth.powerlaw_1m_200k(seed=2, scale=0.005))
    want = [oracle.count(g, threads=4, per_vertex=False).balanced for g in gs]
    return gs, want


def test_batch_matches_oracle_and_replays(gpu_lib, batch_graphs):
    gs, want = batch_graphs
    G = [bbc.Graph.from_synthetic(g) for g in gs]
    try:
        got = bbc.count_batch(G)
        assert got == want
        assert bbc.count_batch(G) == want          # replay of the captured plan
        single = [h.count()[0] for h in G]
        assert single == want
    finally:
        for h in G:
            h.free()


def test_batch_tunings_and_autotune_agree(gpu_lib, batch_graphs):
    gs, want = batch_graphs
    G = [bbc.Graph.from_synthetic(g) for g in gs]
    try:
        for kw in (dict(tile_words=1024, warp_max_wedges=1), dict(warp_max_wedges=512),
                   dict(blocks_per_sm=1), dict(tile_words=4096, split_wedges=200),
                   dict(queue_chunk=1), dict(queue_chunk=64, warp_max_wedges=512),
                   dict(group_warps=8), dict(group_warps=8, blocks_per_sm=1)):
            t = bbc.default_tuning()
            for k, v in kw.items():
                setattr(t, k, v)
            assert bbc.count_batch(G, tuning=t) == want
        best = bbc.autotune_batch(G)
        assert best.tile_words >= 0 and best.blocks_per_sm in (1, 2)
        assert bbc.count_batch(G) == want           # now served with the tuned choice
        assert bbc.count_batch(G, tuning=best) == want
    finally:
        for h in G:
            h.free()


def test_batch_of_one_and_of_none(gpu_lib):
    g = synth.uniform_2k_3k(seed=1)
    G = bbc.Graph.from_synthetic(g)
    try:
        assert bbc.count_batch([G]) == [oracle.count(g, per_vertex=False).balanced]
        assert bbc.count_batch([]) == []
    finally:
        G.free()


# ------------------------------------------------------------------ serving

def test_serving_results_equal_alone_and_in_the_mix(gpu_lib):
    gs = small_batch(120, seed=9)
    gs.insert(7, synth.powerlaw_1m_200k(seed=5, scale=0.02))   # a large request mid-stream
    gs.insert(60, synth.hubs_50k_2m(seed=4, scale=0.002))
    alone = []
    for g in gs:
        G = bbc.Graph.from_synthetic(g)
        alone.append(G.count()[0])
        G.free()
    srv = bbc.Server(8 << 30)
    try:
        tickets = [srv.submit(g) for g in gs]
        got = [srv.wait(t, timeout_s=120.0) for t in tickets]
        assert got == alone
        st = srv.stats()
        assert st["completed"] == len(gs)
        assert 0 < st["p50_us"] <= st["p99_us"]
        # a finished ticket can be polled again
        assert srv.poll(tickets[0]) == alone[0]
    finally:
        srv.close()


def test_serving_errors_stay_with_their_request(gpu_lib):
    lib = gpu_lib
    srv = bbc.Server(8 << 30)
    try:
        ok = synth.uniform_graph(200, 150, 3000, 0.6, seed=1)
        bad = _golden.graph(3, 3, [(0, 0, 1), (5, 1, 1)])          # id out of range
        t_ok1 = srv.submit(ok)
        t_bad = srv.submit(bad)
        t_ok2 = srv.submit(ok)
        want = oracle.count(ok, per_vertex=False).balanced
        assert srv.wait(t_ok1, 60.0) == want
        with pytest.raises(bbc.BBCError) as e:
            srv.wait(t_bad, 60.0)
        assert e.value.status == 2
        assert srv.wait(t_ok2, 60.0) == want
        b = ctypes.c_uint64()
        assert lib.bbc_poll(srv._h, 987654321, ctypes.byref(b)) == 1     # unknown ticket
    finally:
        srv.close()


def test_serving_budget_and_bounded_waits(gpu_lib):
    lib = gpu_lib
    small = bbc.Server(4 << 20)
    try:
        big = synth.uniform_graph(3000, 3000, 200_000, 0.5, seed=2)
        with pytest.raises(bbc.BBCError) as e:
            small.submit(big)
        assert e.value.status == 7
    finally:
        small.close()
    srv = bbc.Server(8 << 30)
    try:
        g = synth.powerlaw_1m_200k(seed=7, scale=0.05)
        t = srv.submit(g)
        b = ctypes.c_uint64()
        st = lib.bbc_wait(srv._h, t, 0, ctypes.byref(b))
        assert st in (0, 9)                                          # done, or timed out
        assert srv.wait(t, 120.0) == oracle.count(g, threads=8, per_vertex=False).balanced
    finally:
        srv.close()


def test_serving_admits_requests_as_memory_frees(gpu_lib):
    """A budget that holds two requests' reservations and 40 requests submitted at once:
    the rest queue, each is admitted only after an earlier one released its memory, the
    reservations never exceed the budget, and every count equals the oracle's."""
    gs = [synth.uniform_graph(1500, 2500, 30_000, 0.7, seed=100 + i) for i in range(40)]
    want = [oracle.count(g, threads=2, per_vertex=False).balanced for g in gs]
    probe = bbc.Server(8 << 30)
    try:
        t = probe.submit(gs[0])
        assert probe.wait(t, 60.0) == want[0]
        reserve = probe.request_info(t)["reserved_bytes"]
    finally:
        probe.close()
    budget = int(2.5 * reserve)
    srv = bbc.Server(budget)
    try:
        tickets = [srv.submit(g) for g in gs]
        got = [srv.wait(t, timeout_s=120.0) for t in tickets]
        assert got == want
        c = srv.counters()
        assert c["submitted"] == c["admitted"] == c["completed"] == len(gs)
        assert c["peak_reserved_bytes"] <= budget == c["budget_bytes"]
        assert c["reserved_bytes"] == 0 and c["queued_now"] == 0
        assert c["max_resident"] <= 2
        # submission is much faster than counting, so most requests found the budget full
        # (a few may arrive after the first completions)
        assert c["max_queued"] >= len(gs) // 2
        assert c["admitted_after_wait"] >= len(gs) // 2
        info = [srv.request_info(t) for t in tickets]
        admit = [q["submit_us"] + q["queued_us"] for q in info]
        done = [q["submit_us"] + q["latency_us"] for q in info]
        for k, q in enumerate(info):
            assert q["status"] == 0 and q["reserved_bytes"] == reserve
            if q["waited_for_memory"]:
                # admitted no earlier than some other request's completion
                assert any(done[j] <= admit[k] + 1.0 for j in range(len(gs)) if j != k), k
        # at no instant were more than two requests admitted and unfinished
        events = sorted([(a, 1) for a in admit] + [(d, -1) for d in done], key=lambda e: (e[0], e[1]))
        live = peak = 0
        for _, step in events:
            live += step
            peak = max(peak, live)
        assert peak <= 2
    finally:
        srv.close()


def test_serving_reservation_covers_measured_peak(gpu_lib):
    """The device memory one request actually reaches at its peak (the library pool's
    high-water mark, preparation temporaries and tick buffers included) stays within the
    reservation that admission charges for it."""
    g = synth.powerlaw_1m_200k(seed=11, scale=0.05)
    srv = bbc.Server(8 << 30)
    try:
        warm = srv.submit(synth.uniform_graph(50, 60, 200, 0.5, seed=1))
        srv.wait(warm, 60.0)
        used0, _ = bbc.memory_usage(reset_high=True)
        t = srv.submit(g)
        assert srv.wait(t, 120.0) == oracle.count(g, threads=8, per_vertex=False).balanced
        _, high = bbc.memory_usage()
        q = srv.request_info(t)
        assert 0 < high - used0 <= q["reserved_bytes"], (high - used0, q["reserved_bytes"])
        assert q["wedges"] > 0 and q["ticks"] >= 1 and q["count_us"] > 0
    finally:
        srv.close()


def test_serving_shutdown_cancels_queued_requests(gpu_lib):
    srv = bbc.Server(8 << 30)
    gs = small_batch(40, seed=12)
    for g in gs:
        srv.submit(g)
    srv.close()   # must return with requests still queued or in flight


_TUNE_SCRIPT = r"""
import json, sys
sys.path.insert(0, {root!r})
from paper_2601_17707_gb300 import bbc, synth
gs = [synth.batch_graph(s) for s in synth.batch_specs(24, seed=31, e_max=20_000)]
G = [bbc.Graph.from_synthetic(g) for g in gs]
out = {{}}
if {tune}:
    out["best"] = bbc.autotune_batch(G).as_dict()
out["used"] = bbc.batch_tuning(G).as_dict()
out["counts"] = bbc.count_batch(G)
print(json.dumps(out))
"""


def test_autotune_choice_persists_across_processes(gpu_lib, tmp_path):
    """One process autotunes a batch with BBC_TUNE_CACHE pointing at a fresh file; a second
    process, given the same file, serves NULL-tuning batch calls of the same shape with
    that choice (bbc_batch_tuning reports it), and its counts equal the oracle's."""
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, BBC_TUNE_CACHE=str(tmp_path / "tune.txt"))

    def run(tune):
        r = subprocess.run([sys.executable, "-c", _TUNE_SCRIPT.format(root=root, tune=tune)],
                           env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        return json.loads(r.stdout.strip().splitlines()[-1])

    first = run(True)
    assert (tmp_path / "tune.txt").exists()
    second = run(False)
    keys = ("tile_words", "warp_max_wedges", "blocks_per_sm", "queue_chunk", "group_warps")
    # the first process serves its own batches with the choice it found ...
    for k in keys:
        assert first["best"][k] in (0, first["used"][k]), k
    # ... and the second process, reading the file, serves them the same way
    assert {k: second["used"][k] for k in keys} == {k: first["used"][k] for k in keys}
    gs = [synth.batch_graph(s) for s in synth.batch_specs(24, seed=31, e_max=20_000)]
    want = [oracle.count(g, per_vertex=False).balanced for g in gs]
    assert first["counts"] == want and second["counts"] == want
