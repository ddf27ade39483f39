"""CPU oracle for balanced-butterfly counting -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package. The library never does, and this package imports nothing
from the library: the two share no code, header, table or helper. Inputs reach both
from the seeded generators, which hold none of the counting arithmetic.

Contents:

* ``count``: the C oracle in ``bbc_oracle.c`` (BB2K's definition, Algorithm 1 of the
  paper, with Lemma 1; dense counters over original ids; optional worker threads).
* ``vertex``: b(x) for a single vertex, from the pair formula on x's own side.
* ``brute_force``: Def. 1 and Def. 2 taken literally -- every (u, w, x, y) 4-tuple is
  tested for presence of all four edges and for an even number of negative edges.
  Pure Python, tiny graphs only.
* ``motif``: the C oracle's sign classes (Sec. VII, Table 7) and balanced
  (2,k)-bicliques (Def. 5) with the pairs on a chosen side.
* ``brute_force_classes`` / ``brute_force_bicliques``: those two taken literally, by
  enumerating 4-tuples (classified by the two centres' sign patterns) and every k-subset
  of a pair's common neighbours (checked for an unbalanced butterfly). Tiny graphs only.
* ``apply_updates`` / ``count_delta``: a batch of edge updates applied to the edge list
  (sign +1 / -1 sets the edge, 0 deletes it) and the change of both counts, by counting
  the graph before and after with ``count``.
* ``matrix_counts``: the signed/unsigned co-occurrence identity with a library
  matmul (numpy float64 BLAS; exact, since every product and partial sum is an
  integer of magnitude at most |V| < 2^53, then converted to int64). For the signed biadjacency A (entries +1, -1, 0) and
  M = |A|, with c = M M^T and s = A A^T over pairs u < w of side U:
  unsigned butterflies = sum C(c_uw, 2), and balanced - unbalanced =
  sum (s_uw^2 - c_uw) / 2 (each pair of common neighbours contributes the product of
  its four signs). Per vertex of U the same sums are taken over the row of u.
"""

from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bbc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict[int, ctypes.CDLL] = {}

STATUS = {0: "ok", 1: "bad input", 2: "no memory", 3: "overflow"}


def lib_path(mutant: int = 0) -> str:
    name = "libbbc_oracle.so" if mutant == 0 else f"libbbc_oracle_mutant{mutant}.so"
    return os.path.join(_BUILD, name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Compiles the C oracle (gcc, -O2) and returns the path of the shared object."""
    out = lib_path(mutant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", f"-DBBCO_MUTANT={mutant}",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _lib(mutant: int = 0) -> ctypes.CDLL:
    with _LOCK:
        if mutant not in _LIBS:
            lib = ctypes.CDLL(build(mutant))
            i32, i64, p = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
            lib.bbco_count.argtypes = [i32, i32, i64, p, p, p, ctypes.c_int, ctypes.c_int,
                                       p, p, p, p]
            lib.bbco_count.restype = ctypes.c_int
            lib.bbco_count_sample.argtypes = [i32, i32, i64, p, p, p, ctypes.c_int, ctypes.c_int,
                                              i64, i64, p, p, p, p, p]
            lib.bbco_count_sample.restype = ctypes.c_int
            lib.bbco_vertex.argtypes = [i32, i32, i64, p, p, p, ctypes.c_int, i32, p]
            lib.bbco_vertex.restype = ctypes.c_int
            lib.bbco_motif.argtypes = [i32, i32, i64, p, p, p, ctypes.c_int, ctypes.c_uint32,
                                       ctypes.c_int, p]
            lib.bbco_motif.restype = ctypes.c_int
            lib.bbco_mutant.restype = ctypes.c_int
            _LIBS[mutant] = lib
        return _LIBS[mutant]


def _arrays(g):
    u = np.ascontiguousarray(g.u, dtype=np.int32)
    v = np.ascontiguousarray(g.v, dtype=np.int32)
    s = np.ascontiguousarray(g.sign, dtype=np.int8)
    return u, v, s


@dataclass
class Counts:
    balanced: int
    unbalanced: int
    per_u: np.ndarray | None
    per_v: np.ndarray | None


def count(g, orient_low: bool = False, threads: int = 1, per_vertex: bool = True,
          mutant: int = 0) -> Counts:
    """Balanced / unbalanced butterflies (and per-vertex balanced counts) of ``g``.

    ``g`` has fields n_u, n_v, u, v, sign (edge list, signs +1/-1, no duplicates).
    """
    lib = _lib(mutant)
    u, v, s = _arrays(g)
    b = ctypes.c_uint64(0)
    ub = ctypes.c_uint64(0)
    pu = np.zeros(g.n_u, dtype=np.uint64) if per_vertex else None
    pv = np.zeros(g.n_v, dtype=np.uint64) if per_vertex else None
    st = lib.bbco_count(g.n_u, g.n_v, u.shape[0], u.ctypes.data, v.ctypes.data, s.ctypes.data,
                        int(orient_low), int(threads), ctypes.addressof(b), ctypes.addressof(ub),
                        pu.ctypes.data if pu is not None else None,
                        pv.ctypes.data if pv is not None else None)
    if st != 0:
        raise ValueError(f"oracle: {STATUS.get(st, st)}")
    return Counts(int(b.value), int(ub.value), pu, pv)


def count_sample(g, stride: int, offset: int = 0, threads: int = 1, per_vertex: bool = True):
    """The oracle over the anchors offset, offset + stride, ... of U only (a bounded
    sample of the full count, for timing). Returns (Counts, oriented wedges visited)."""
    lib = _lib(0)
    u, v, s = _arrays(g)
    b = ctypes.c_uint64(0)
    ub = ctypes.c_uint64(0)
    w = ctypes.c_uint64(0)
    pu = np.zeros(g.n_u, dtype=np.uint64) if per_vertex else None
    pv = np.zeros(g.n_v, dtype=np.uint64) if per_vertex else None
    st = lib.bbco_count_sample(g.n_u, g.n_v, u.shape[0], u.ctypes.data, v.ctypes.data,
                               s.ctypes.data, 0, int(threads), int(offset), int(stride),
                               ctypes.addressof(b), ctypes.addressof(ub),
                               pu.ctypes.data if pu is not None else None,
                               pv.ctypes.data if pv is not None else None, ctypes.addressof(w))
    if st != 0:
        raise ValueError(f"oracle: {STATUS.get(st, st)}")
    return Counts(int(b.value), int(ub.value), pu, pv), int(w.value)


def vertex(g, side: int, x: int, mutant: int = 0) -> int:
    """b(x) for vertex ``x`` of side ``side`` (0 = U, 1 = V), from x's own side."""
    lib = _lib(mutant)
    u, v, s = _arrays(g)
    out = ctypes.c_uint64(0)
    st = lib.bbco_vertex(g.n_u, g.n_v, u.shape[0], u.ctypes.data, v.ctypes.data, s.ctypes.data,
                         int(side), int(x), ctypes.addressof(out))
    if st != 0:
        raise ValueError(f"oracle: {STATUS.get(st, st)}")
    return int(out.value)


CLASS_NAMES = ("coherent ++/++", "coherent ++/--", "coherent --/--", "incoherent +-/+-",
               "mixed ++/+-", "mixed +-/--")


def _side(g, side: int):
    """The edge arrays with the pair side first (side 0 = U, 1 = V)."""
    u, v, s = _arrays(g)
    if side == 0:
        return g.n_u, g.n_v, u, v, s
    return g.n_v, g.n_u, v, u, s


def motif(g, kind: str, k: int = 2, side: int = 0, threads: int = 1, mutant: int = 0) -> tuple:
    """kind "classes": the six sign-class totals in CLASS_NAMES order; kind "biclique":
    (balanced (2,k)-bicliques, all (2,k)-bicliques). ``side`` holds the pair (the "2")."""
    lib = _lib(mutant)
    n_a, n_b, a, b, s = _side(g, side)
    kind_id = {"classes": 1, "biclique": 2}[kind]
    out = (ctypes.c_uint64 * 6)()
    st = lib.bbco_motif(n_a, n_b, a.shape[0], a.ctypes.data, b.ctypes.data, s.ctypes.data,
                        kind_id, int(k), int(threads), ctypes.addressof(out))
    if st != 0:
        raise ValueError(f"oracle: {STATUS.get(st, st)}")
    return tuple(int(x) for x in out[:6 if kind_id == 1 else 2])


def _sign_map(g, side: int):
    n_a, n_b, a, b, s = _side(g, side)
    return n_a, n_b, {(x, y): z for x, y, z in zip(a.tolist(), b.tolist(), s.tolist())}


def brute_force_classes(g, side: int = 0) -> tuple:
    """Every (u<w on the pair side, x<y on the other) 4-tuple with all four edges, put in
    the class named by its two centres' sign patterns. Tiny graphs only."""
    n_a, n_b, sign = _sign_map(g, side)
    if n_a * n_b > 400:
        raise ValueError("brute force is for graphs with |U|*|V| <= 400")

    def kind(u, w, x):          # 0: both +, 1: both -, 2: the signs differ
        su, sw = sign[(u, x)], sign[(w, x)]
        return 2 if su != sw else (0 if su > 0 else 1)

    index = {(0, 0): 0, (0, 1): 1, (1, 1): 2, (2, 2): 3, (0, 2): 4, (1, 2): 5}
    out = [0] * 6
    for u, w in itertools.combinations(range(n_a), 2):
        for x, y in itertools.combinations(range(n_b), 2):
            if all(e in sign for e in ((u, x), (u, y), (w, x), (w, y))):
                out[index[tuple(sorted((kind(u, w, x), kind(u, w, y))))]] += 1
    return tuple(out)


def brute_force_bicliques(g, k: int, side: int = 0) -> tuple:
    """(balanced, all) (2,k)-bicliques by enumeration: each k-subset of a pair's common
    neighbours is a (2,k)-biclique, balanced when none of its butterflies holds an odd
    number of negative edges (Def. 5 with Def. 2). Tiny graphs only."""
    n_a, n_b, sign = _sign_map(g, side)
    if n_a * n_b > 400:
        raise ValueError("brute force is for graphs with |U|*|V| <= 400")
    bal = total = 0
    for u, w in itertools.combinations(range(n_a), 2):
        common = [x for x in range(n_b) if (u, x) in sign and (w, x) in sign]
        for sub in itertools.combinations(common, k):
            total += 1
            if all(sign[(u, x)] * sign[(u, y)] * sign[(w, x)] * sign[(w, y)] > 0
                   for x, y in itertools.combinations(sub, 2)):
                bal += 1
    return bal, total


@dataclass
class EdgeList:
    n_u: int
    n_v: int
    u: np.ndarray
    v: np.ndarray
    sign: np.ndarray


def apply_updates(g, u, v, new_sign) -> EdgeList:
    """The graph after setting edge (u[i], v[i]) to new_sign[i] (0 deletes it). Raises on a
    pair repeated in the batch or a deletion of an absent edge."""
    edges = {(a, b): s for a, b, s in zip(np.asarray(g.u).tolist(), np.asarray(g.v).tolist(),
                                          np.asarray(g.sign).tolist())}
    seen = set()
    for a, b, s in zip(np.asarray(u).tolist(), np.asarray(v).tolist(), np.asarray(new_sign).tolist()):
        if (a, b) in seen:
            raise ValueError("update batch repeats an edge")
        seen.add((a, b))
        if s == 0:
            if (a, b) not in edges:
                raise ValueError("deletion of an absent edge")
            del edges[(a, b)]
        else:
            edges[(a, b)] = s
    keys = sorted(edges)
    return EdgeList(g.n_u, g.n_v, np.array([k[0] for k in keys], dtype=np.int32),
                    np.array([k[1] for k in keys], dtype=np.int32),
                    np.array([edges[k] for k in keys], dtype=np.int8))


def count_delta(g, u, v, new_sign, threads: int = 1) -> tuple:
    """(B(G') - B(G), Ub(G') - Ub(G)) for the batch, by two full counts."""
    before = count(g, threads=threads, per_vertex=False)
    after = count(apply_updates(g, u, v, new_sign), threads=threads, per_vertex=False)
    return after.balanced - before.balanced, after.unbalanced - before.unbalanced


def brute_force(g) -> Counts:
    """Def. 1 / Def. 2 literally: test every u<w in U, x<y in V. Tiny graphs only."""
    if g.n_u * g.n_v > 400:
        raise ValueError("brute force is for graphs with |U|*|V| <= 400")
    sign = {}
    for a, b, s in zip(np.asarray(g.u).tolist(), np.asarray(g.v).tolist(),
                       np.asarray(g.sign).tolist()):
        sign[(a, b)] = s
    bal = unb = 0
    per_u = [0] * g.n_u
    per_v = [0] * g.n_v
    for u1, u2 in itertools.combinations(range(g.n_u), 2):
        for x, y in itertools.combinations(range(g.n_v), 2):
            edges = [(u1, x), (u1, y), (u2, x), (u2, y)]
            if not all(e in sign for e in edges):
                continue
            negatives = sum(1 for e in edges if sign[e] < 0)
            if negatives % 2 == 0:
                bal += 1
                per_u[u1] += 1
                per_u[u2] += 1
                per_v[x] += 1
                per_v[y] += 1
            else:
                unb += 1
    return Counts(bal, unb, np.array(per_u, dtype=np.uint64), np.array(per_v, dtype=np.uint64))


def _gram(a: np.ndarray) -> np.ndarray:
    """a @ a.T for an integer matrix with entries in {-1, 0, 1}, exactly, as int64."""
    f = a.astype(np.float64)
    return np.rint(f @ f.T).astype(np.int64)


def matrix_counts(g, per_vertex: bool = False) -> Counts:
    """Balanced / unbalanced counts from dense co-occurrence matrices (numpy matmul)."""
    a = np.zeros((g.n_u, g.n_v), dtype=np.int64)
    a[np.asarray(g.u, dtype=np.int64), np.asarray(g.v, dtype=np.int64)] = np.asarray(g.sign, dtype=np.int64)
    m = np.abs(a)
    c = _gram(m)
    s = _gram(a)
    np.fill_diagonal(c, 0)
    np.fill_diagonal(s, 0)
    unsigned_pairs = c * (c - 1) // 2          # butterflies per ordered pair (u, w), u != w
    signed_pairs = (s * s - c) // 2            # (balanced - unbalanced) per pair
    bal_pairs = (unsigned_pairs + signed_pairs) // 2
    unb_pairs = (unsigned_pairs - signed_pairs) // 2
    bal = int(np.triu(bal_pairs, 1).sum())
    unb = int(np.triu(unb_pairs, 1).sum())
    per_u = per_v = None
    if per_vertex:
        per_u = bal_pairs.sum(axis=1).astype(np.uint64)
        at = np.ascontiguousarray(a.T)
        ct = _gram(np.abs(at))
        st = _gram(at)
        np.fill_diagonal(ct, 0)
        np.fill_diagonal(st, 0)
        per_v = ((ct * (ct - 1) // 2 + (st * st - ct) // 2) // 2).sum(axis=1).astype(np.uint64)
    return Counts(bal, unb, per_u, per_v)


def unsigned_butterflies(g) -> int:
    """Unsigned butterfly count sum_{u<w} C(c_uw, 2) via a library matmul."""
    a = np.zeros((g.n_u, g.n_v), dtype=np.int64)
    a[np.asarray(g.u, dtype=np.int64), np.asarray(g.v, dtype=np.int64)] = 1
    c = _gram(a)
    np.fill_diagonal(c, 0)
    return int(np.triu(c * (c - 1) // 2, 1).sum())
