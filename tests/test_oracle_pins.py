"""Pins of the CPU oracle against facts fixed by the paper and by the mathematics.

Every test here runs on the CPU. None of them re-types the oracle's formula: each
compares it with something else -- the paper's figures, the definition enumerated
literally, closed forms, a library matmul identity, or invariances of the problem.
"""

from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_2601_17707_gb300 import synth
from tests import _golden


def _random_graph(rng, n_u, n_v, density, p_pos=0.5):
    mask = rng.random((n_u, n_v)) < density
    uu, vv = np.nonzero(mask)
    sign = np.where(rng.random(uu.shape[0]) < p_pos, 1, -1)
    return _golden.graph(n_u, n_v, list(zip(uu.tolist(), vv.tolist(), sign.tolist())))


def _edges(g):
    return list(zip(g.u.tolist(), g.v.tolist(), g.sign.tolist()))


def _assert_same(a, b):
    assert a.balanced == b.balanced
    assert a.unbalanced == b.unbalanced
    np.testing.assert_array_equal(a.per_u, b.per_u)
    np.testing.assert_array_equal(a.per_v, b.per_v)


# ------------------------------------------------------------------ paper figures

def test_fig2_single_butterflies():
    """Fig. 2: (a)-(e) balanced, (f)-(g) unbalanced."""
    cases = _golden.load_cases("fig2_butterflies.txt")
    assert [c[0] for c in cases] == list("abcdefg")
    for name, g, label in cases:
        got = oracle.count(g)
        want = (1, 0) if label == "balanced" else (0, 1)
        assert (got.balanced, got.unbalanced) == want, name
        bf = oracle.brute_force(g)
        assert (bf.balanced, bf.unbalanced) == want, name


@pytest.mark.parametrize("name", ["fig1b_signed_k44.txt", "fig9_drug_target.txt"])
def test_paper_figure_graphs(name):
    g, expect = _golden.load(name)
    got = oracle.count(g)
    assert got.balanced == expect["balanced"]
    assert got.unbalanced == expect["unbalanced"]
    assert got.per_u.tolist() == expect["per_u"]
    assert got.per_v.tolist() == expect["per_v"]
    _assert_same(got, oracle.brute_force(g))


# ------------------------------------------------------------------ brute force

@pytest.mark.parametrize("a,b", [(2, 2), (2, 3), (3, 2), (3, 3)])
def test_every_sign_pattern_of_small_complete_graphs(a, b):
    pairs = [(i, j) for i in range(a) for j in range(b)]
    for mask in range(1 << len(pairs)):
        edges = [(i, j, -1 if (mask >> k) & 1 else 1) for k, (i, j) in enumerate(pairs)]
        g = _golden.graph(a, b, edges)
        _assert_same(oracle.count(g), oracle.brute_force(g))


def test_random_tiny_graphs_against_brute_force():
    rng = np.random.default_rng(1)
    for trial in range(300):
        n_u = int(rng.integers(1, 11))
        n_v = int(rng.integers(1, 11))
        g = _random_graph(rng, n_u, n_v, float(rng.uniform(0.2, 0.95)), float(rng.uniform(0.1, 0.9)))
        want = oracle.brute_force(g)
        _assert_same(oracle.count(g), want)
        _assert_same(oracle.count(g, orient_low=True), want)


# ------------------------------------------------------------------ closed forms

@pytest.mark.parametrize("a,b", [(2, 2), (3, 5), (7, 4), (12, 9), (40, 31)])
def test_complete_bipartite_closed_forms(a, b):
    full = [(i, j, 1) for i in range(a) for j in range(b)]
    g = _golden.graph(a, b, full)
    got = oracle.count(g)
    assert got.balanced == math.comb(a, 2) * math.comb(b, 2)
    assert got.unbalanced == 0
    assert got.per_u.tolist() == [(a - 1) * math.comb(b, 2)] * a
    assert got.per_v.tolist() == [(b - 1) * math.comb(a, 2)] * b
    # all edges negative: the same as all positive (switching every vertex of V)
    neg = oracle.count(_golden.graph(a, b, [(i, j, -1) for i, j, _ in full]))
    _assert_same(neg, got)
    # one negative edge: (a-1)(b-1) butterflies contain it and become unbalanced
    one = [(i, j, -1 if (i, j) == (a - 1, b - 1) else 1) for i, j, _ in full]
    got1 = oracle.count(_golden.graph(a, b, one))
    assert got1.unbalanced == (a - 1) * (b - 1)
    assert got1.balanced == math.comb(a, 2) * math.comb(b, 2) - (a - 1) * (b - 1)


def test_empty_and_degenerate_graphs():
    assert oracle.count(_golden.graph(0, 0, [])).balanced == 0
    g = _golden.graph(5, 4, [])
    got = oracle.count(g)
    assert (got.balanced, got.unbalanced) == (0, 0)
    assert got.per_u.tolist() == [0] * 5 and got.per_v.tolist() == [0] * 4
    star = _golden.graph(1, 50, [(0, j, 1) for j in range(50)])  # a star has no 4-cycle
    assert oracle.count(star).balanced == 0
    single = _golden.graph(3, 3, [(1, 2, -1)])
    assert oracle.count(single).balanced == 0


# ------------------------------------------------------------------ library identities

def test_matrix_identity_full_uniform_workload():
    """|U|=2,000, |V|=3,000, 20,000 edges: exact agreement with int64 matmul identities."""
    g = synth.uniform_2k_3k(seed=0)
    got = oracle.count(g)
    want = oracle.matrix_counts(g)
    assert got.balanced == want.balanced and got.unbalanced == want.unbalanced
    assert got.balanced + got.unbalanced == oracle.unsigned_butterflies(g)
    assert got.balanced > 0


def test_matrix_identity_per_vertex():
    rng = np.random.default_rng(7)
    for _ in range(6):
        g = _random_graph(rng, int(rng.integers(20, 70)), int(rng.integers(20, 70)),
                          float(rng.uniform(0.05, 0.5)), float(rng.uniform(0.2, 0.9)))
        got = oracle.count(g)
        want = oracle.matrix_counts(g, per_vertex=True)
        assert (got.balanced, got.unbalanced) == (want.balanced, want.unbalanced)
        np.testing.assert_array_equal(got.per_u, want.per_u)
        np.testing.assert_array_equal(got.per_v, want.per_v)


# ------------------------------------------------------------------ invariances

def _transpose(g):
    return _golden.graph(g.n_v, g.n_u, list(zip(g.v.tolist(), g.u.tolist(), g.sign.tolist())))


def test_side_and_orientation_agreement():
    g = synth.powerlaw_1m_200k(seed=3, scale=0.002)
    a = oracle.count(g)
    b = oracle.count(_transpose(g))
    assert (a.balanced, a.unbalanced) == (b.balanced, b.unbalanced)
    np.testing.assert_array_equal(a.per_u, b.per_v)
    np.testing.assert_array_equal(a.per_v, b.per_u)
    _assert_same(a, oracle.count(g, orient_low=True))
    assert int(a.per_u.sum()) == 2 * a.balanced == int(a.per_v.sum())


def test_switching_invariance():
    """Negating every edge at one vertex changes no butterfly's balance."""
    rng = np.random.default_rng(11)
    g = synth.powerlaw_1m_200k(seed=5, scale=0.002)
    base = oracle.count(g)
    for side, n in ((0, g.n_u), (1, g.n_v)):
        for x in rng.integers(0, n, size=4).tolist():
            hit = (g.u == x) if side == 0 else (g.v == x)
            s2 = np.where(hit, -g.sign, g.sign).astype(np.int8)
            h = _golden.graph(g.n_u, g.n_v, list(zip(g.u.tolist(), g.v.tolist(), s2.tolist())))
            _assert_same(oracle.count(h), base)


def test_relabel_shuffle_and_union():
    rng = np.random.default_rng(2)
    g = synth.powerlaw_1m_200k(seed=9, scale=0.002)
    base = oracle.count(g)
    pu = rng.permutation(g.n_u)
    pv = rng.permutation(g.n_v)
    order = rng.permutation(g.u.shape[0])
    h = _golden.graph(g.n_u, g.n_v, list(zip(pu[g.u][order].tolist(), pv[g.v][order].tolist(),
                                                g.sign[order].tolist())))
    got = oracle.count(h)
    assert (got.balanced, got.unbalanced) == (base.balanced, base.unbalanced)
    np.testing.assert_array_equal(got.per_u[pu], base.per_u)
    np.testing.assert_array_equal(got.per_v[pv], base.per_v)
    # disjoint union: counts add, per-vertex arrays concatenate
    k = synth.uniform_graph(300, 200, 3000, 0.6, seed=4)
    kc = oracle.count(k)
    edges = _edges(g) + [(a + g.n_u, b + g.n_v, s) for a, b, s in _edges(k)]
    un = oracle.count(_golden.graph(g.n_u + k.n_u, g.n_v + k.n_v, edges))
    assert un.balanced == base.balanced + kc.balanced
    assert un.unbalanced == base.unbalanced + kc.unbalanced
    np.testing.assert_array_equal(un.per_u, np.concatenate([base.per_u, kc.per_u]))
    np.testing.assert_array_equal(un.per_v, np.concatenate([base.per_v, kc.per_v]))


def test_planted_factions_without_flips_are_fully_balanced():
    """Signs +1 inside a faction and -1 across are switching-equivalent to all +1."""
    g = synth.chung_lu_graph(500, 20000, 100000, 1.8, 2.5, 10000, 500, seed=1, factions_flip=0.0)
    got = oracle.count(g, threads=4)
    assert got.unbalanced == 0
    assert got.balanced == oracle.unsigned_butterflies(g)


def test_iid_sign_statistics_band():
    """E[balanced / all] = (1 + (2q-1)^4) / 2 for i.i.d. signs with P(+) = q (a sanity band)."""
    g = synth.uniform_graph(300, 400, 24000, 0.7, seed=2)
    got = oracle.count(g, per_vertex=False)
    frac = got.balanced / (got.balanced + got.unbalanced)
    assert abs(frac - (1 + 0.4 ** 4) / 2) < 0.02


# ------------------------------------------------------------------ per-vertex

def test_single_vertex_function_matches_full_pass():
    rng = np.random.default_rng(3)
    g = _random_graph(rng, 40, 55, 0.3, 0.6)
    full = oracle.count(g)
    assert [oracle.vertex(g, 0, x) for x in range(g.n_u)] == full.per_u.tolist()
    assert [oracle.vertex(g, 1, x) for x in range(g.n_v)] == full.per_v.tolist()
    h = synth.powerlaw_1m_200k(seed=1, scale=0.002)
    fh = oracle.count(h)
    for x in rng.integers(0, h.n_u, size=5).tolist():
        assert oracle.vertex(h, 0, x) == int(fh.per_u[x])
    for x in rng.integers(0, h.n_v, size=5).tolist():
        assert oracle.vertex(h, 1, x) == int(fh.per_v[x])


def test_threads_agree():
    g = synth.powerlaw_1m_200k(seed=2, scale=0.003)
    _assert_same(oracle.count(g, threads=1), oracle.count(g, threads=6))


def test_rejects_bad_input():
    with pytest.raises(ValueError):
        oracle.count(_golden.graph(2, 2, [(0, 2, 1)]))
    with pytest.raises(ValueError):
        oracle.count(_golden.graph(2, 2, [(0, 1, 0)]))


# ------------------------------------------------------------------ sensitivity

def _pin_failures(mutant):
    """Runs a compact set of the pins above against a mutant build; returns what failed."""
    failed = []
    for name in ("fig1b_signed_k44.txt", "fig9_drug_target.txt"):
        g, e = _golden.load(name)
        c = oracle.count(g, mutant=mutant)
        if (c.balanced, c.unbalanced, c.per_u.tolist(), c.per_v.tolist()) != (
                e["balanced"], e["unbalanced"], e["per_u"], e["per_v"]):
            failed.append(name)
    for name, g, label in _golden.load_cases("fig2_butterflies.txt"):
        c = oracle.count(g, mutant=mutant)
        if (c.balanced, c.unbalanced) != ((1, 0) if label == "balanced" else (0, 1)):
            failed.append("fig2" + name)
    k = _golden.graph(5, 4, [(i, j, 1) for i in range(5) for j in range(4)])
    c = oracle.count(k, mutant=mutant)
    if c.balanced != math.comb(5, 2) * math.comb(4, 2) or c.per_v.tolist() != [3 * 10] * 4:
        failed.append("closed form")
    rng = np.random.default_rng(5)
    for _ in range(20):
        g = _random_graph(rng, 6, 7, 0.6, 0.5)
        c = oracle.count(g, mutant=mutant)
        b = oracle.brute_force(g)
        if (c.balanced, c.unbalanced) != (b.balanced, b.unbalanced) or \
                c.per_u.tolist() != b.per_u.tolist() or c.per_v.tolist() != b.per_v.tolist():
            failed.append("brute force")
            break
    return failed


def test_pins_pass_on_the_oracle():
    assert _pin_failures(0) == []


@pytest.mark.parametrize("mutant", range(1, 8))
def test_each_planted_mistake_fails_a_pin(mutant):
    assert oracle._lib(mutant).bbco_mutant() == mutant
    assert _pin_failures(mutant), f"mutant {mutant} passed every pin"


def test_anchor_samples_partition_the_count():
    """Strided anchor samples with offsets 0..k-1 add up to the full count."""
    g = synth.powerlaw_1m_200k(seed=6, scale=0.002)
    full = oracle.count(g, per_vertex=False)
    tot_b = tot_u = tot_w = 0
    for off in range(3):
        c, w = oracle.count_sample(g, stride=3, offset=off, threads=2, per_vertex=False)
        tot_b += c.balanced
        tot_u += c.unbalanced
        tot_w += w
    assert (tot_b, tot_u) == (full.balanced, full.unbalanced)
    dv = np.bincount(g.v, minlength=g.n_v).astype(np.int64)
    assert tot_w == int((dv * (dv - 1) // 2).sum())  # every oriented wedge exactly once
