"""The seeded input generators against the recipe they state (CPU only).

The generators feed both the oracle and the CUDA path, so a drift in them would change
every workload silently. These tests hold them to their stated definitions: SplitMix64
in counter mode (Steele, Lea and Flood, OOPSLA 2014), the offset power-law expected
degrees, the first |E| distinct pairs in draw order, seeded determinism, and the ranges
of the batched workload.
"""

from __future__ import annotations

import math

import numpy as np
import pytest

from paper_2601_17707_gb300 import synth

GOLDEN = 0x9E3779B97F4A7C15


def test_splitmix64_known_answers():
    # the first outputs of SplitMix64 from state 1234567, as printed with its public
    # reference implementations: state += golden gamma, then the finaliser
    state = np.uint64(1234567)
    with np.errstate(over="ignore"):
        z = synth._mix(state + np.arange(1, 6, dtype=np.uint64) * np.uint64(GOLDEN))
    assert [int(x) for x in z] == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                                   4593380528125082431, 16408922859458223821]


def test_counter_mode_windows_and_uniforms():
    full = synth.splitmix_u64(7, synth.TAG_U, 0, 64)
    assert np.array_equal(full[10:30], synth.splitmix_u64(7, synth.TAG_U, 10, 20))
    # streams of other tags and seeds differ
    assert not np.array_equal(full, synth.splitmix_u64(7, synth.TAG_V, 0, 64))
    assert not np.array_equal(full, synth.splitmix_u64(8, synth.TAG_U, 0, 64))
    r = synth.uniform01(7, synth.TAG_U, 0, 100_000)
    assert r.min() >= 0.0 and r.max() < 1.0
    k = r * 2.0 ** 53
    assert np.array_equal(k, np.floor(k))          # 53-bit grid
    assert abs(r.mean() - 0.5) < 0.005 and abs(r.var() - 1 / 12) < 0.002


@pytest.mark.parametrize("n,e,gamma,dmax", [(1000, 20_000, 2.2, 500.0), (50_000, 2_000_000, 1.8, 40_000.0),
                                            (200, 5_000, 2.5, 200.0)])
def test_powerlaw_weights_follow_the_offset_power_law(n, e, gamma, dmax):
    w = synth.powerlaw_weights(n, e, gamma, dmax)
    assert w.shape == (n,)
    assert w.sum() == pytest.approx(e, rel=1e-9)
    assert w[0] == pytest.approx(dmax, rel=1e-12)
    assert np.all(np.diff(w) < 0)
    # w_1 / w_0 = (i0 / (1 + i0))^(1 / (gamma - 1)) fixes i0; every other term follows
    q = (w[1] / w[0]) ** (gamma - 1.0)
    i0 = q / (1.0 - q)
    i = np.arange(n, dtype=np.float64)
    assert np.allclose(w, dmax * (i0 / (i + i0)) ** (1.0 / (gamma - 1.0)), rtol=1e-8)


def test_infeasible_degree_sequences_are_refused():
    with pytest.raises(ValueError):
        synth.powerlaw_weights(10, 1000, 2.2, 50.0)
    with pytest.raises(ValueError):
        synth.uniform_graph(3, 3, 10, 0.5)


def _first_distinct_by_scan(seed, n_u, n_v, n_edges, cdf_u=None, cdf_v=None):
    """One pass over the draw sequence, keeping the first n_edges distinct pairs."""
    kept, seen, i = [], set(), 0
    while len(kept) < n_edges:
        ru = synth.uniform01(seed, synth.TAG_U, i, 1)[0]
        rv = synth.uniform01(seed, synth.TAG_V, i, 1)[0]
        u = min(int(ru * n_u), n_u - 1) if cdf_u is None else min(int(np.searchsorted(cdf_u, ru, "right")), n_u - 1)
        v = min(int(rv * n_v), n_v - 1) if cdf_v is None else min(int(np.searchsorted(cdf_v, rv, "right")), n_v - 1)
        if (u, v) not in seen:
            seen.add((u, v))
            kept.append((u, v))
        i += 1
    return sorted(kept)


def test_uniform_graph_is_the_first_distinct_pairs_in_draw_order():
    # dense enough that many draws repeat (600 of 1,200 pairs), so several rounds run
    g = synth.uniform_graph(40, 30, 600, 0.7, seed=3)
    got = list(zip(g.u.tolist(), g.v.tolist()))
    assert got == _first_distinct_by_scan(3, 40, 30, 600)
    assert set(np.unique(g.sign).tolist()) <= {-1, 1}
    assert g.u.dtype == np.int32 and g.v.dtype == np.int32 and g.sign.dtype == np.int8


def test_chung_lu_graph_is_the_first_distinct_pairs_in_draw_order():
    n_u, n_v, e = 60, 45, 700
    g = synth.chung_lu_graph(n_u, n_v, e, 2.2, 2.2, 40.0, 40.0, 0.8, seed=5)
    cu = synth._cdf(synth.powerlaw_weights(n_u, e, 2.2, 40.0))
    cv = synth._cdf(synth.powerlaw_weights(n_v, e, 2.2, 40.0))
    got = list(zip(g.u.tolist(), g.v.tolist()))
    assert got == _first_distinct_by_scan(5, n_u, n_v, e, cu, cv)


def test_named_uniform_workload_shape_and_determinism():
    g = synth.uniform_2k_3k(0)
    assert (g.n_u, g.n_v, g.n_edges) == (2000, 3000, 20_000)
    keys = g.u.astype(np.int64) * g.n_v + g.v
    assert np.all(np.diff(keys) > 0)                 # distinct and sorted by (u, v)
    assert 0.68 < float((g.sign == 1).mean()) < 0.72  # P(+) = 0.7, 6 standard deviations
    h = synth.uniform_2k_3k(0)
    assert np.array_equal(g.u, h.u) and np.array_equal(g.v, h.v) and np.array_equal(g.sign, h.sign)
    assert not np.array_equal(g.v, synth.uniform_2k_3k(1).v)


def test_factions_without_flips_sign_by_faction_agreement():
    g = synth.chung_lu_graph(300, 200, 3000, 2.2, 2.2, 100.0, 100.0, seed=2, factions_flip=0.0)
    # a +1 edge joins equal factions, a -1 edge different ones: the signs must be
    # consistent with a two-colouring of the vertices, i.e. around every cycle the
    # product of signs is +1. Propagate colours over a spanning forest and check all edges.
    col_u = np.full(g.n_u, -1)
    col_v = np.full(g.n_v, -1)
    adj_u = [[] for _ in range(g.n_u)]
    adj_v = [[] for _ in range(g.n_v)]
    for k, (a, b) in enumerate(zip(g.u.tolist(), g.v.tolist())):
        adj_u[a].append(k)
        adj_v[b].append(k)
    for root in range(g.n_u):
        if col_u[root] >= 0 or not adj_u[root]:
            continue
        col_u[root] = 0
        stack = [("u", root)]
        while stack:
            side, x = stack.pop()
            for k in (adj_u[x] if side == "u" else adj_v[x]):
                a, b, s = int(g.u[k]), int(g.v[k]), int(g.sign[k])
                if side == "u" and col_v[b] < 0:
                    col_v[b] = col_u[a] if s == 1 else 1 - col_u[a]
                    stack.append(("v", b))
                elif side == "v" and col_u[a] < 0:
                    col_u[a] = col_v[b] if s == 1 else 1 - col_v[b]
                    stack.append(("u", a))
    same = col_u[g.u] == col_v[g.v]
    assert np.array_equal(same, g.sign == 1)


def test_shuffle_keeps_the_edge_multiset():
    g = synth.uniform_graph(100, 80, 2000, 0.6, seed=4)
    s = synth.shuffled(g, seed=9)
    assert not np.array_equal(g.u, s.u) or not np.array_equal(g.v, s.v)
    a = sorted(zip(g.u.tolist(), g.v.tolist(), g.sign.tolist()))
    b = sorted(zip(s.u.tolist(), s.v.tolist(), s.sign.tolist()))
    assert a == b


def test_batch_specs_follow_their_ranges():
    specs = synth.batch_specs(4096, seed=0)
    assert len(specs) == 4096
    assert len({s.seed for s in specs}) == 4096
    for s in specs:
        assert 100 <= s.n_u <= 50_000 and 100 <= s.n_v <= 50_000
        assert 1 <= s.n_edges <= min(500_000, s.n_u * s.n_v // 4)
        cap = max(2, s.n_edges // 10)
        assert s.dmax_u == min(s.n_v, 50_000, cap) and s.dmax_v == min(s.n_u, 50_000, cap)
        assert 0.5 <= s.p_pos <= 0.95
    # log-uniform sizes: about half the draws fall below the geometric midpoint
    mid = math.sqrt(100 * 50_000)
    frac = np.mean([s.n_u < mid for s in specs])
    assert 0.45 < frac < 0.55


def test_batch_members_do_not_depend_on_the_worker_count():
    specs = sorted(synth.batch_specs(256, seed=1), key=lambda s: s.n_edges)[:8]
    one = synth.batch_graphs(specs, workers=1)
    two = synth.batch_graphs(specs, workers=2)
    for a, b in zip(one, two):
        assert np.array_equal(a.u, b.u) and np.array_equal(a.v, b.v) and np.array_equal(a.sign, b.sign)
