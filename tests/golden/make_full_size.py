"""Writes the expected counts of the full-size synthetic workloads, from the CPU oracle.

Usage: python tests/golden/make_full_size.py <workload> [threads]

The only counting code this script runs is ``oracle.count`` (the plain CPU oracle); the
graph comes from the seeded generators. The output file holds the workload name, the
seed, a SHA-256 digest of the generated edge list (so a test can confirm it generated
the same graph), the balanced and unbalanced totals, and SHA-256 digests of the
per-vertex arrays (little-endian uint64, original vertex ids).
"""

from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2601_17707_gb300 import synth  # noqa: E402


def edge_digest(g) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.u, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(g.v, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(g.sign, dtype="i1").tobytes())
    return h.hexdigest()


def array_digest(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<u8").tobytes()).hexdigest()


def main() -> None:
    name = sys.argv[1]
    threads = int(sys.argv[2]) if len(sys.argv) > 2 else (os.cpu_count() or 1)
    seed = 0
    g = synth.WORKLOADS[name](seed=seed)
    t0 = time.time()
    c = oracle.count(g, threads=threads, per_vertex=True)
    dt = time.time() - t0
    out = os.path.join(HERE, f"full_{name}.txt")
    with open(out, "w") as f:
        f.write(f"# Expected counts of the synthetic workload '{name}' (seed {seed}), written by\n")
        f.write("# tests/golden/make_full_size.py from the CPU oracle alone "
                f"({threads} threads, {dt:.0f} s).\n")
        f.write(f"workload {name}\nseed {seed}\n")
        f.write(f"n_u {g.n_u}\nn_v {g.n_v}\nn_edges {g.n_edges}\n")
        f.write(f"edges_sha256 {edge_digest(g)}\n")
        f.write(f"balanced {c.balanced}\nunbalanced {c.unbalanced}\n")
        f.write(f"per_u_sha256 {array_digest(c.per_u)}\nper_v_sha256 {array_digest(c.per_v)}\n")
        f.write(f"per_u_sum {int(c.per_u.sum())}\nper_v_sum {int(c.per_v.sum())}\n")
    print(out, dt)


if __name__ == "__main__":
    main()
