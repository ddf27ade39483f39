"""Seeded synthetic signed bipartite graphs.

This module only draws inputs. It holds none of the counting arithmetic, so that the
CPU oracle and the CUDA path can both be fed from it without sharing any step of the
method. Everything is a pure function of ``(config, seed)``.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used in counter mode: draw ``i`` of
stream ``tag`` is the SplitMix64 finaliser applied to
``key(seed, tag) + (i + 1) * 0x9E3779B97F4A7C15``. A 53-bit uniform in [0, 1) is
``(z >> 11) * 2**-53``.

Graph families (the paper's datasets, Table 2 of Sec. VI, are not available; these
stand in for them with the shapes the workload description fixes):

* ``uniform``: ``|E|`` distinct (u, v) pairs drawn uniformly, each sign +1 with
  probability ``p_pos``.
* ``chung_lu``: per side, expected degrees follow an offset power law
  ``w_i = d_max * (i0 / (i + i0)) ** (1 / (gamma - 1))`` with ``i0`` solved so that
  ``sum(w) = |E|``. Endpoints are drawn with probability proportional to ``w`` on
  each side, and draws repeat until exactly ``|E|`` distinct pairs exist (the first
  ``|E|`` distinct pairs in draw order are kept).
* ``factions``: Chung-Lu topology; every vertex joins one of two factions with
  probability 1/2; an edge is +1 inside a faction and -1 across; each sign is then
  flipped with probability ``flip``.

Edges are returned sorted by (u, v) unless ``shuffle`` is requested.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream tags keep the draws of different purposes independent.
TAG_U = 1
TAG_V = 2
TAG_SIGN = 3
TAG_FACTION_U = 4
TAG_FACTION_V = 5
TAG_FLIP = 6
TAG_SHUFFLE = 7
TAG_BATCH = 8


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _key(seed: int, tag: int) -> np.uint64:
    base = np.array([(int(seed) * 0x100000001B3 + int(tag) * 0x9E3779B1) & 0xFFFFFFFFFFFFFFFF],
                    dtype=np.uint64)
    return _mix(base)[0]


def splitmix_u64(seed: int, tag: int, start: int, count: int) -> np.ndarray:
    """Draws ``start .. start+count-1`` of stream ``(seed, tag)`` as uint64."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
        return _mix(_key(seed, tag) + idx * _GOLDEN)


def uniform01(seed: int, tag: int, start: int, count: int) -> np.ndarray:
    """53-bit uniforms in [0, 1) from stream ``(seed, tag)``."""
    z = splitmix_u64(seed, tag, start, count)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def powerlaw_weights(n: int, n_edges: int, gamma: float, d_max: float) -> np.ndarray:
    """Offset power-law expected degrees ``w_i = d_max (i0/(i+i0))^(1/(gamma-1))``.

    ``i0`` is found by bisection so that ``sum(w) == n_edges`` (to 1e-9 relative).
    """
    a = 1.0 / (gamma - 1.0)
    i = np.arange(n, dtype=np.float64)

    def total(i0: float) -> float:
        return float(np.sum(d_max * (i0 / (i + i0)) ** a))

    if n * d_max < n_edges:
        raise ValueError("infeasible degree sequence: n * d_max < |E|")
    lo, hi = 1e-9, 1.0
    while total(hi) < n_edges:
        hi *= 2.0
        if hi > 1e18:
            raise ValueError("could not bracket i0")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if total(mid) < n_edges:
            lo = mid
        else:
            hi = mid
        if hi - lo <= 1e-12 * hi:
            break
    i0 = 0.5 * (lo + hi)
    return d_max * (i0 / (i + i0)) ** a


@dataclass
class SignedBipartite:
    """A signed bipartite graph as an edge list (ids are 0-based per side)."""

    n_u: int
    n_v: int
    u: np.ndarray  # int32[E]
    v: np.ndarray  # int32[E]
    sign: np.ndarray  # int8[E], +1 or -1
    name: str = ""

    @property
    def n_edges(self) -> int:
        return int(self.u.shape[0])


def _draw_distinct_pairs(seed: int, n_u: int, n_v: int, n_edges: int,
                         cdf_u: np.ndarray | None, cdf_v: np.ndarray | None) -> np.ndarray:
    """First ``n_edges`` distinct pairs (as keys u * n_v + v) in draw order, then sorted."""
    if n_edges > n_u * n_v:
        raise ValueError("more edges than vertex pairs")
    keys_parts: list[np.ndarray] = []
    drawn = 0
    have = np.empty(0, dtype=np.int64)
    while True:
        need = n_edges - have.shape[0]
        if need <= 0:
            break
        batch = max(int(need * 1.15) + 1024, 4096)
        ru = uniform01(seed, TAG_U, drawn, batch)
        rv = uniform01(seed, TAG_V, drawn, batch)
        if cdf_u is None:
            uu = np.minimum((ru * n_u).astype(np.int64), n_u - 1)
        else:
            uu = np.minimum(np.searchsorted(cdf_u, ru, side="right"), n_u - 1).astype(np.int64)
        if cdf_v is None:
            vv = np.minimum((rv * n_v).astype(np.int64), n_v - 1)
        else:
            vv = np.minimum(np.searchsorted(cdf_v, rv, side="right"), n_v - 1).astype(np.int64)
        drawn += batch
        keys_parts.append(uu * n_v + vv)
        allk = np.concatenate(keys_parts)
        keys_parts = [allk]
        uniq, first = np.unique(allk, return_index=True)
        if uniq.shape[0] >= n_edges:
            order = np.sort(first)[:n_edges]
            have = np.sort(allk[order])
            break
        have = uniq
        # keep the raw draw order list (keys_parts) and continue drawing
    return have


def _cdf(w: np.ndarray) -> np.ndarray:
    c = np.cumsum(w)
    return c / c[-1]


def uniform_graph(n_u: int, n_v: int, n_edges: int, p_pos: float, seed: int = 0) -> SignedBipartite:
    keys = _draw_distinct_pairs(seed, n_u, n_v, n_edges, None, None)
    u = (keys // n_v).astype(np.int32)
    v = (keys % n_v).astype(np.int32)
    r = uniform01(seed, TAG_SIGN, 0, n_edges)
    sign = np.where(r < p_pos, 1, -1).astype(np.int8)
    return SignedBipartite(n_u, n_v, u, v, sign, name="uniform")


def chung_lu_graph(n_u: int, n_v: int, n_edges: int, gamma_u: float, gamma_v: float,
                   dmax_u: float, dmax_v: float, p_pos: float = 0.5, seed: int = 0,
                   factions_flip: float | None = None) -> SignedBipartite:
    wu = powerlaw_weights(n_u, n_edges, gamma_u, dmax_u)
    wv = powerlaw_weights(n_v, n_edges, gamma_v, dmax_v)
    keys = _draw_distinct_pairs(seed, n_u, n_v, n_edges, _cdf(wu), _cdf(wv))
    u = (keys // n_v).astype(np.int32)
    v = (keys % n_v).astype(np.int32)
    if factions_flip is None:
        r = uniform01(seed, TAG_SIGN, 0, n_edges)
        sign = np.where(r < p_pos, 1, -1).astype(np.int8)
        name = "chung_lu"
    else:
        fu = uniform01(seed, TAG_FACTION_U, 0, n_u) < 0.5
        fv = uniform01(seed, TAG_FACTION_V, 0, n_v) < 0.5
        same = fu[u] == fv[v]
        flip = uniform01(seed, TAG_FLIP, 0, n_edges) < factions_flip
        pos = same ^ flip
        sign = np.where(pos, 1, -1).astype(np.int8)
        name = "factions"
    return SignedBipartite(n_u, n_v, u, v, sign, name=name)


def shuffled(g: SignedBipartite, seed: int = 0) -> SignedBipartite:
    """The same graph with its edge list in a seeded random order."""
    keys = splitmix_u64(seed, TAG_SHUFFLE, 0, g.n_edges)
    order = np.argsort(keys, kind="stable")
    return SignedBipartite(g.n_u, g.n_v, g.u[order], g.v[order], g.sign[order], name=g.name)


# ---------------------------------------------------------------------------------
# The named workloads.

def uniform_2k_3k(seed: int = 0) -> SignedBipartite:
    """|U|=2,000, |V|=3,000, 20,000 distinct uniform pairs, P(+)=0.7."""
    g = uniform_graph(2000, 3000, 20000, 0.7, seed)
    g.name = "uniform_2k_3k_20k"
    return g


def powerlaw_1m_200k(seed: int = 0, scale: float = 1.0) -> SignedBipartite:
    """Chung-Lu, |U|=1e6, |V|=2e5, |E|=2e7, gamma 2.2 both sides, d_max 50,000, P(+)=0.8.

    ``scale`` < 1 shrinks every size (vertices, edges, d_max) by the same factor, for
    tests that need the same shape at a size a CPU finishes quickly.
    """
    n_u = max(int(1_000_000 * scale), 2)
    n_v = max(int(200_000 * scale), 2)
    n_e = max(int(20_000_000 * scale), 1)
    dmax = max(50_000 * scale, 2.0)
    g = chung_lu_graph(n_u, n_v, n_e, 2.2, 2.2, min(dmax, n_v), min(dmax, n_u), 0.8, seed)
    g.name = "powerlaw_1m_200k_20m" if scale == 1.0 else f"powerlaw_1m_200k_20m_x{scale:g}"
    return g


def hubs_50k_2m(seed: int = 0, scale: float = 1.0) -> SignedBipartite:
    """|U|=5e4 (gamma 1.8, top ~1e6), |V|=2e6 (gamma 2.5, d_max |U|), |E|=1e8, factions, flip 0.1."""
    n_u = max(int(50_000 * scale), 2)
    n_v = max(int(2_000_000 * scale), 2)
    n_e = max(int(100_000_000 * scale), 1)
    g = chung_lu_graph(n_u, n_v, n_e, 1.8, 2.5, min(1_000_000 * scale, n_v), n_u,
                       seed=seed, factions_flip=0.1)
    g.name = "hubs_50k_2m_100m" if scale == 1.0 else f"hubs_50k_2m_100m_x{scale:g}"
    return g


@dataclass
class BatchGraphSpec:
    n_u: int
    n_v: int
    n_edges: int
    dmax_u: float
    dmax_v: float
    p_pos: float
    seed: int


def batch_specs(n_graphs: int = 4096, seed: int = 0, e_max: int = 500_000) -> list[BatchGraphSpec]:
    """Per-graph shapes of the batched workload.

    |U|, |V| log-uniform in [100, 50,000]; |E| log-uniform in [1,000, e_max] capped at
    |U||V|/4; per side d_max = min(other side, 50,000, floor(|E|/10)); P(+) ~ U(0.5, 0.95).
    Graph g draws its edges with seed ``seed * 1_000_003 + g + 1``.
    """
    r = uniform01(seed, TAG_BATCH, 0, 4 * n_graphs).reshape(n_graphs, 4)
    lo, hi = math.log(100.0), math.log(50_000.0)
    specs = []
    for g in range(n_graphs):
        n_u = int(round(math.exp(lo + (hi - lo) * r[g, 0])))
        n_v = int(round(math.exp(lo + (hi - lo) * r[g, 1])))
        elo, ehi = math.log(1000.0), math.log(float(e_max))
        n_e = int(round(math.exp(elo + (ehi - elo) * r[g, 2])))
        n_e = max(1, min(n_e, (n_u * n_v) // 4))
        cap = max(2, n_e // 10)
        dmax_u = float(min(n_v, 50_000, cap))
        dmax_v = float(min(n_u, 50_000, cap))
        p_pos = 0.5 + 0.45 * float(r[g, 3])
        specs.append(BatchGraphSpec(n_u, n_v, n_e, dmax_u, dmax_v, p_pos, seed * 1_000_003 + g + 1))
    return specs


def batch_graph(spec: BatchGraphSpec) -> SignedBipartite:
    g = chung_lu_graph(spec.n_u, spec.n_v, spec.n_edges, 2.2, 2.2, spec.dmax_u, spec.dmax_v,
                       spec.p_pos, spec.seed)
    g.name = "batch_member"
    return g


def large_serving_graph(seed: int = 0) -> SignedBipartite:
    """The 1% large request of the serving mix: |U|=2e5, |V|=1e5, |E|=5e6, gamma 2.2, P(+)=0.8."""
    g = chung_lu_graph(200_000, 100_000, 5_000_000, 2.2, 2.2, 50_000, 50_000, 0.8, seed)
    g.name = "serve_large_200k_100k_5m"
    return g


WORKLOADS = {
    "uniform_2k_3k_20k": uniform_2k_3k,
    "powerlaw_1m_200k_20m": powerlaw_1m_200k,
    "hubs_50k_2m_100m": hubs_50k_2m,
}
