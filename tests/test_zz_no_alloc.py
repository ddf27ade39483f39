"""The allocation-free entry point, bbc_count_noalloc, against bbc_count.

bbc_count_noalloc serves callers that cannot allocate device memory when they count
(inside stream capture, in latency-critical loops, or when another allocator already
holds all device memory). It keeps its scratch in one static device array, so these
tests check that two calls in a row both agree exactly with bbc_count (counts are
integers: zero tolerance), that the calls leave free device memory unchanged, and that
a graph beyond the array's limit is refused. This file is collected last on purpose.
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
