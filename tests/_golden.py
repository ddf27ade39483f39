"""Reader for the small text fixtures under tests/golden/."""

from __future__ import annotations

import os
from types import SimpleNamespace

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _graph(n_u, n_v, edges):
    return SimpleNamespace(
        n_u=n_u, n_v=n_v,
        u=np.array([e[0] for e in edges], dtype=np.int32),
        v=np.array([e[1] for e in edges], dtype=np.int32),
        sign=np.array([e[2] for e in edges], dtype=np.int8),
    )


def _sign(tok):
    return {"+": 1, "-": -1}[tok]


def load(name):
    """Returns (graph, expectations) for a single-graph fixture."""
    n_u = n_v = 0
    edges = []
    expect = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "n_u":
                n_u = int(t[1])
            elif t[0] == "n_v":
                n_v = int(t[1])
            elif t[0] == "edge":
                edges.append((int(t[1]), int(t[2]), _sign(t[3])))
            elif t[0] == "expect":
                vals = [int(x) for x in t[2:]]
                expect[t[1]] = vals[0] if len(vals) == 1 else vals
    return _graph(n_u, n_v, edges), expect


def load_cases(name):
    """Returns [(case_name, graph, label)] for a multi-case fixture (2x2 butterflies)."""
    cases = []
    cur = None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "case":
                cur = [t[1], [], t[2]]
                cases.append(cur)
            elif t[0] == "edge":
                cur[1].append((int(t[1]), int(t[2]), _sign(t[3])))
    return [(c[0], _graph(2, 2, c[1]), c[2]) for c in cases]


def graph(n_u, n_v, edges):
    return _graph(n_u, n_v, edges)


def load_batch(name="batch_4096_chung_lu.txt"):
    """The oracle-written totals of the batched workload: (header dict, list of
    (n_u, n_v, n_edges, balanced, unbalanced) per member in index order)."""
    head, rows = {}, []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "g":
                assert int(t[1]) == len(rows)
                rows.append(tuple(int(x) for x in t[2:7]))
            else:
                head[t[0]] = t[1]
    return head, rows


def load_full(name):
    """The oracle-written facts of a full-size workload (tests/golden/full_<name>.txt)."""
    out = {}
    with open(os.path.join(GOLDEN, f"full_{name}.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split()
            out[k] = v
    return out
