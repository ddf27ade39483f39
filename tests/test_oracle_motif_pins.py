"""Pins of the oracle's motif counts (sign classes of Sec. VII / Table 7, balanced
(2,k)-bicliques of Def. 5): literal enumeration, closed forms, identities with the
butterfly count, a symmetry, the Fig. 9 hand enumeration, overflow, and planted mistakes.
All CPU.
"""

from __future__ import annotations

import itertools
import math

import numpy as np
import pytest

import oracle
from tests import _golden


def _random_graph(rng, n_u, n_v, density, p_pos):
    edges = [(a, b, 1 if rng.random() < p_pos else -1)
             for a in range(n_u) for b in range(n_v) if rng.random() < density]
    return _golden.graph(n_u, n_v, edges)


def _k(n_u, n_v, neg=()):
    return _golden.graph(n_u, n_v, [(a, b, -1 if (a, b) in neg else 1)
                                    for a in range(n_u) for b in range(n_v)])


@pytest.mark.parametrize("side", [0, 1])
def test_classes_equal_enumeration(side):
    rng = np.random.default_rng(11)
    for _ in range(40):
        g = _random_graph(rng, int(rng.integers(2, 9)), int(rng.integers(2, 9)), 0.6, 0.55)
        assert oracle.motif(g, "classes", side=side, threads=3) == \
            oracle.brute_force_classes(g, side=side)


def test_classes_every_sign_pattern_of_small_bicliques():
    for n_u, n_v in ((2, 2), (2, 3), (3, 3)):
        cells = [(a, b) for a in range(n_u) for b in range(n_v)]
        for mask in range(1 << len(cells)):
            neg = {c for i, c in enumerate(cells) if mask >> i & 1}
            g = _k(n_u, n_v, neg)
            for side in (0, 1):
                assert oracle.motif(g, "classes", side=side) == \
                    oracle.brute_force_classes(g, side=side)


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_bicliques_equal_enumeration(k):
    rng = np.random.default_rng(100 + k)
    for _ in range(25):
        g = _random_graph(rng, int(rng.integers(2, 8)), int(rng.integers(3, 10)), 0.7, 0.6)
        for side in (0, 1):
            assert oracle.motif(g, "biclique", k=k, side=side, threads=2) == \
                oracle.brute_force_bicliques(g, k, side=side)


def test_identities_with_the_butterfly_count():
    """Coherent + incoherent = balanced and mixed = unbalanced (Lemma 1); the six classes
    add up to the unsigned count (a library matmul); (2,2)-bicliques are butterflies."""
    rng = np.random.default_rng(3)
    for _ in range(15):
        g = _random_graph(rng, 12, 15, 0.5, 0.7)
        cl = oracle.motif(g, "classes")
        c = oracle.count(g, per_vertex=False)
        assert sum(cl[:4]) == c.balanced and cl[4] + cl[5] == c.unbalanced
        assert sum(cl) == oracle.unsigned_butterflies(g)
        assert oracle.motif(g, "biclique", k=2) == (c.balanced, c.balanced + c.unbalanced)


def test_global_negation_swaps_the_sign_classes():
    rng = np.random.default_rng(4)
    for _ in range(10):
        g = _random_graph(rng, 10, 9, 0.6, 0.6)
        h = _golden.graph(g.n_u, g.n_v, list(zip(g.u.tolist(), g.v.tolist(),
                                                 (-g.sign.astype(int)).tolist())))
        a, b = oracle.motif(g, "classes"), oracle.motif(h, "classes")
        assert (b[0], b[1], b[2], b[3], b[4], b[5]) == (a[2], a[1], a[0], a[3], a[5], a[4])


@pytest.mark.parametrize("m,k", [(6, 2), (7, 3), (9, 4), (12, 6)])
def test_closed_forms_on_k2m(m, k):
    """K_{2,m} all positive: every centre is pp. One negative edge at (0, 0): that centre
    is asymmetric, the other m - 1 stay pp."""
    g = _k(2, m)
    assert oracle.motif(g, "classes") == (math.comb(m, 2), 0, 0, 0, 0, 0)
    assert oracle.motif(g, "biclique", k=k) == (math.comb(m, k), math.comb(m, k))
    h = _k(2, m, neg={(0, 0)})
    assert oracle.motif(h, "classes") == (math.comb(m - 1, 2), 0, 0, 0, m - 1, 0)
    assert oracle.motif(h, "biclique", k=k) == (math.comb(m - 1, k), math.comb(m, k))
    # the side matters for k > 2: from side V every pair of centres has 2 common
    # neighbours, so (2,k)-bicliques with k > 2 do not exist there
    assert oracle.motif(g, "biclique", k=3, side=1) == (0, 0)


def test_fig9_drug_target_classes():
    g, e = _golden.load("fig9_drug_target.txt")
    assert list(oracle.motif(g, "classes", side=0)) == e["classes_u"]


def test_overflow_is_reported():
    g = _k(2, 200)
    with pytest.raises(ValueError, match="overflow"):
        oracle.motif(g, "biclique", k=100)              # C(200, 100) > 2^64
    assert oracle.motif(g, "biclique", k=199) == (200, 200)


def _motif_pin_failures(mutant):
    failed = []
    g, e = _golden.load("fig9_drug_target.txt")
    if list(oracle.motif(g, "classes", mutant=mutant)) != e["classes_u"]:
        failed.append("fig9 classes")
    for m, k in ((6, 2), (7, 3), (9, 4)):
        if oracle.motif(_k(2, m), "biclique", k=k, mutant=mutant) != (math.comb(m, k),) * 2:
            failed.append("closed form")
    rng = np.random.default_rng(9)
    for _ in range(10):
        h = _random_graph(rng, 6, 7, 0.6, 0.5)
        if oracle.motif(h, "classes", mutant=mutant) != oracle.brute_force_classes(h):
            failed.append("classes enumeration")
            break
    return failed


def test_motif_pins_pass_on_the_oracle():
    assert _motif_pin_failures(0) == []


@pytest.mark.parametrize("mutant", [8, 9])
def test_each_planted_motif_mistake_fails_a_pin(mutant):
    assert oracle._lib(mutant).bbco_mutant() == mutant
    assert _motif_pin_failures(mutant), f"mutant {mutant} passed every motif pin"
