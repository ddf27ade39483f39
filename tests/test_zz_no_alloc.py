"""The allocation-free entry point, bbc_count_noalloc, against bbc_count.

bbc_count_noalloc serves callers that cannot allocate device memory when they count
(another framework's allocator already holds all device memory, or a latency-critical
loop must not pay for cudaMalloc's synchronisation). It keeps its scratch in one static
device array, so these tests check that two calls in a row both agree exactly with
bbc_count (counts are integers: zero tolerance), that the calls leave free device memory
unchanged, and that a graph beyond the array's limit is refused. One graph sits near the
limit with hubs whose counts need 16- and 32-bit counters over several tiles. This file
is collected last on purpose.
"""

from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2601_17707_gb300 import bbc, synth

pytestmark = pytest.mark.gpu


def _noalloc(lib, G, totals):
    return lib.bbc_count_noalloc(G.handle, totals.data_ptr(), torch.cuda.current_stream().cuda_stream)


def test_two_calls_in_a_row_match_bbc_count(gpu_lib):
    lib = gpu_lib
    for g in (synth.powerlaw_1m_200k(seed=11, scale=0.01), synth.uniform_2k_3k(seed=0)):
        G = bbc.Graph.from_synthetic(g)
        try:
            want = G.count()[:2]
            totals = torch.full((2,), -1, dtype=torch.int64, device="cuda")
            _noalloc(lib, G, totals)  # first call on the device does the address look-up
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            for _ in range(2):
                totals.fill_(-1)
                assert _noalloc(lib, G, totals) == 0, bbc.last_error()
                torch.cuda.synchronize()
                got = totals.cpu().numpy().view(np.uint64).tolist()
                assert tuple(int(x) for x in got) == want
            assert torch.cuda.mem_get_info()[0] == free_before
        finally:
            G.free()


def _wide_hub_graph():
    """65,000 pair-side vertices (just under the 65,520 limit) over 70,000 centres: vertex
    0 on every centre and vertex 1 on 66,000 of them share more than 65,535 centres (32-bit
    counters, several tiles each), 200 vertices on 300 centres each share more than 255
    centres with the hubs (16-bit counters), and the rest have four centres each."""
    rng = np.random.default_rng(5)
    n_u, n_v = 65_000, 70_000
    us = [np.zeros(n_v, np.int64), np.ones(66_000, np.int64)]
    vs = [np.arange(n_v), np.arange(66_000)]
    mid = rng.choice(np.arange(2, n_u), size=200, replace=False)
    for x in mid:
        us.append(np.full(300, x))
        vs.append(rng.choice(n_v, size=300, replace=False))
    rest = np.setdiff1d(np.arange(2, n_u), mid)
    us.append(np.repeat(rest, 4))
    vs.append(rng.integers(0, n_v, size=4 * rest.size))
    key = np.unique(np.concatenate(us) * n_v + np.concatenate(vs))
    u = (key // n_v).astype(np.int32)
    v = (key % n_v).astype(np.int32)
    s = np.where(rng.random(key.size) < 0.7, 1, -1).astype(np.int8)
    return synth.SignedBipartite(n_u, n_v, u, v, s)


def test_wide_tiles_and_counter_widths_match_bbc_count(gpu_lib):
    lib = gpu_lib
    g = _wide_hub_graph()
    G = bbc.Graph.from_synthetic(g, flags=bbc.SIDE_FORCE_U)
    try:
        want = G.count()[:2]
        assert want[0] > 0 and want[1] > 0
        totals = torch.full((2,), -1, dtype=torch.int64, device="cuda")
        for _ in range(2):
            totals.fill_(-1)
            assert _noalloc(lib, G, totals) == 0, bbc.last_error()
            torch.cuda.synchronize()
            got = tuple(int(x) for x in totals.cpu().numpy().view(np.uint64).tolist())
            assert got == want
    finally:
        G.free()


def test_graph_beyond_the_static_scratch_is_refused(gpu_lib):
    lib = gpu_lib
    n_u = 70_000
    u = np.repeat(np.arange(n_u, dtype=np.int32), 2)
    v = np.tile(np.array([0, 1], dtype=np.int32), n_u)
    s = np.ones(u.shape[0], dtype=np.int8)
    g = synth.SignedBipartite(n_u, 2, u, v, s)
    G = bbc.Graph.from_synthetic(g, flags=bbc.SIDE_FORCE_U)
    try:
        totals = torch.zeros(2, dtype=torch.int64, device="cuda")
        assert _noalloc(lib, G, totals) == 1
        assert "at most 65520" in bbc.last_error()
    finally:
        G.free()
