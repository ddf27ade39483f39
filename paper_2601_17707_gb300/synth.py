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


class _InverseCdf:
    """searchsorted(cdf, r, side="right") for many r at once, through a table of bucket
    starts: bucket b = floor(r * 2^22) holds the answer between tab[b] and tab[b + 1], so
    a few vectorised bisection steps finish it. The result equals numpy's searchsorted."""

    BITS = 22

    def __init__(self, cdf: np.ndarray):
        self.cdf = cdf
        k = 1 << self.BITS
        self.tab = np.searchsorted(cdf, np.arange(k + 1, dtype=np.float64) / k, side="right")

    def __call__(self, r: np.ndarray) -> np.ndarray:
        b = (r * (1 << self.BITS)).astype(np.int64)
        lo = self.tab[b]
        hi = self.tab[b + 1]
        n = self.cdf.shape[0]
        while True:
            open_ = lo < hi
            if not open_.any():
                return lo
            mid = (lo + hi) >> 1
            go = np.zeros(lo.shape, dtype=bool)
            m = open_
            go[m] = self.cdf[np.minimum(mid[m], n - 1)] <= r[m]
            lo = np.where(m & go, mid + 1, lo)
            hi = np.where(m & ~go, mid, hi)


def _draw_distinct_pairs(seed: int, n_u: int, n_v: int, n_edges: int,
                         cdf_u: np.ndarray | None, cdf_v: np.ndarray | None) -> np.ndarray:
    """First ``n_edges`` distinct pairs (as keys u * n_v + v) in draw order, then sorted.

    Draws come in rounds; each round's keys are de-duplicated among themselves (first
    occurrence wins) and against the pairs already kept, so the result is the same as
    scanning the whole draw sequence once.
    """
    if n_edges > n_u * n_v:
        raise ValueError("more edges than vertex pairs")
    # the bucket table pays off only for many draws over a long table
    big = n_edges >= (1 << 20)
    inv_u = (_InverseCdf(cdf_u) if big else (lambda r: np.searchsorted(cdf_u, r, side="right"))) \
        if cdf_u is not None else None
    inv_v = (_InverseCdf(cdf_v) if big else (lambda r: np.searchsorted(cdf_v, r, side="right"))) \
        if cdf_v is not None else None
    kept = np.empty(0, dtype=np.int64)      # sorted distinct keys so far
    drawn = 0
    fresh_ratio = 1.0                        # sizes the next round; does not change the result
    while kept.shape[0] < n_edges:
        need = n_edges - kept.shape[0]
        batch = max(int(need * 1.15 / max(fresh_ratio, 0.02)) + 1024, 4096)
        ru = uniform01(seed, TAG_U, drawn, batch)
        rv = uniform01(seed, TAG_V, drawn, batch)
        if cdf_u is None:
            uu = np.minimum((ru * n_u).astype(np.int64), n_u - 1)
        else:
            uu = np.minimum(inv_u(ru), n_u - 1).astype(np.int64)
        if cdf_v is None:
            vv = np.minimum((rv * n_v).astype(np.int64), n_v - 1)
        else:
            vv = np.minimum(inv_v(rv), n_v - 1).astype(np.int64)
        drawn += batch
        keys = uu * n_v + vv
        uniq, first = np.unique(keys, return_index=True)
        if kept.shape[0]:
            pos = np.searchsorted(kept, uniq)
            pos[pos == kept.shape[0]] = 0
            fresh = kept[pos] != uniq
            uniq, first = uniq[fresh], first[fresh]
        fresh_ratio = uniq.shape[0] / batch
        if uniq.shape[0] > need:
            # keep the fresh keys whose first draw comes before the need-th fresh first draw
            is_first = np.zeros(batch, dtype=bool)
            is_first[first] = True
            cutoff = int(np.searchsorted(np.cumsum(is_first), need))  # draw index of the need-th
            uniq = uniq[first <= cutoff]
        kept = np.insert(kept, np.searchsorted(kept, uniq), uniq) if kept.shape[0] else uniq
    return kept


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
    "serve_large_200k_100k_5m": large_serving_graph,
}


def _batch_worker(spec: BatchGraphSpec) -> SignedBipartite:
    return batch_graph(spec)


def batch_graphs(specs: list[BatchGraphSpec], workers: int | None = None) -> list[SignedBipartite]:
    """Generates many batch members, in a pool of worker processes when workers > 1.

    The pool uses the 'spawn' start method, so it is safe in processes that already
    initialised CUDA. Every graph is a pure function of its spec, so the result does not
    depend on the number of workers.
    """
    import os

    workers = workers if workers is not None else min(16, os.cpu_count() or 1)
    if workers <= 1 or len(specs) < 8:
        return [batch_graph(s) for s in specs]
    import concurrent.futures as cf
    import multiprocessing as mp

    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_batch_worker, specs, chunksize=max(1, len(specs) // (4 * workers))))
